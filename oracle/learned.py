"""Learned correction of the block-OSRC preconditioner (oracle side).

Test infrastructure only (imported by tests, never by the product).  The
paper has no learned part; this is the reading the library implements:

* Preconditioner (linear in r): z = P r + C r with P the block-OSRC operator
  (Eq. 19) and C a local stencil: for dof m of block i and its 4 RWG
  neighbours q (the other edges of the two triangles of Gamma_i that share
  edge m, ascending local dof index), with sources s in {r, P r},
      z_D[m] += sum_{q, s} a[q,s,DD] s_D[q] + a[q,s,DN] s_N[q]
      z_N[m] += sum_{q, s} a[q,s,ND] s_D[q] + a[q,s,NN] s_N[q]
  (q = 0 is m itself; complex coefficients a, 5 x 2 x 4 per dof).
* The coefficients of every dof come from a small network of its geometry:
  features (10): k_i l_m, rho_i, 1 for the exterior block, k_i l_q of the 4
  neighbours (same order), k_i^2 (A_1 + A_2) of its two triangles, the cosine
  between their normals, and 1 if the two triangles lie on different
  interfaces (a junction edge); network x -> relu(W1 x + b1) -> relu(W2 h1 +
  b2) -> W3 h2 + b3 with 80 outputs, the (re, im) parts of a in the order
  [q][s][DD, DN, ND, NN][re, im].  Parameters are augmented matrices [W | b]
  row-major, layer after layer (W1: H x 11, W2: H x (H+1), W3: 80 x (H+1)).
* Parametrisations of the coefficients: a table (the coefficients are the
  parameters) or the network above.
* Training objective (power loss), for vectors z and a centre c0:
      L = mean_z ||E^K z||^2 / ||z||^2,   E = I - M (P + C) / c0,
  the error propagator of Richardson's iteration with step 1 / c0 taken K
  times; over vectors with E[z z^H] = I it estimates ||E^K||_F^2 / n, i.e.
  sum_i |1 - lambda_i / c0|^(2K) / n for normal E.  c0 is the mean Rayleigh
  quotient <z, M P z> / <z, z> of the plain preconditioned operator.

Everything here is plain FP64 numpy written from these definitions.
"""
from __future__ import annotations

import numpy as np

from .skeleton import Skeleton

N_FEAT = 10
N_OUT = 80


def neighbours(sk: Skeleton, i: int) -> np.ndarray:
    """(N_i, 4) local dofs of the other edges of the two triangles of each dof."""
    D = sk.dof[i]
    nb = [set() for _ in range(sk.N[i])]
    for t in range(len(D)):
        for a in range(3):
            for b in range(3):
                if a != b:
                    nb[D[t, a]].add(int(D[t, b]))
    out = np.zeros((sk.N[i], 4), dtype=np.int64)
    for m in range(sk.N[i]):
        lst = sorted(nb[m])
        if len(lst) != 4:
            raise ValueError("an RWG dof of a closed surface has exactly 4 neighbours")
        out[m] = lst
    return out


def _edge_lengths(sk: Skeleton, i: int) -> np.ndarray:
    E = sk.edges[i]
    return np.linalg.norm(sk.V[E[:, 1]] - sk.V[E[:, 0]], axis=1)


def features(sk: Skeleton, k, rho) -> np.ndarray:
    """Geometric features (rows, 10), rows in the global dof order."""
    rows = []
    for i in range(sk.n_domains):
        nb = neighbours(sk, i)
        le = _edge_lengths(sk, i)
        ki = float(np.real(k[i]))
        tris = sk.tris[i]
        nrm = sk.swap[i][:, None] * sk.normal[tris]       # normals of Gamma_i's triangles as oriented in block i
        area = sk.area[tris]
        # interface of every triangle of block i: the neighbouring domain
        other = np.where(sk.L[tris, 0] == i, sk.L[tris, 1], sk.L[tris, 0])
        x = np.zeros((sk.N[i], N_FEAT))
        x[:, 0] = ki * le
        x[:, 1] = float(np.real(rho[i]))
        x[:, 2] = 1.0 if i == 0 else 0.0
        x[:, 3:7] = ki * le[nb]
        for m in range(sk.N[i]):
            t = np.where((sk.dof[i] == m).any(axis=1))[0]
            x[m, 7] = ki * ki * (area[t[0]] + area[t[1]])
            x[m, 8] = float(nrm[t[0]] @ nrm[t[1]])
            x[m, 9] = 1.0 if other[t[0]] != other[t[1]] else 0.0
        rows.append(x)
    return np.concatenate(rows, axis=0)


def param_shapes(H: int):
    return [(H, N_FEAT + 1), (H, H + 1), (N_OUT, H + 1)]


def n_params(H: int) -> int:
    return sum(a * b for a, b in param_shapes(H))


def unpack(theta: np.ndarray, H: int):
    mats, o = [], 0
    for a, b in param_shapes(H):
        mats.append(np.asarray(theta[o:o + a * b], dtype=np.float64).reshape(a, b))
        o += a * b
    return mats


def forward(theta, H, X):
    """Outputs (rows, 80) and the activations needed by backward."""
    W1, W2, W3 = unpack(theta, H)
    h1 = np.maximum(X @ W1[:, :-1].T + W1[:, -1], 0.0)
    h2 = np.maximum(h1 @ W2[:, :-1].T + W2[:, -1], 0.0)
    return h2 @ W3[:, :-1].T + W3[:, -1], (h1, h2)


def loss_grad(theta, H, X, T, w):
    """L = sum_rows w_row |y - t|^2 and dL/dtheta (same layout as theta)."""
    W1, W2, W3 = unpack(theta, H)
    y, (h1, h2) = forward(theta, H, X)
    d = y - T
    L = float(np.sum(w[:, None] * d * d))
    g3 = 2.0 * w[:, None] * d
    return L, backward(theta, H, X, (h1, h2), g3)


def backward(theta, H, X, acts, g3):
    """dL/dtheta from dL/dy (rows, 80) after forward."""
    W1, W2, W3 = unpack(theta, H)
    h1, h2 = acts
    dW3 = np.concatenate([g3.T @ h2, g3.sum(0)[:, None]], axis=1)
    g2 = (g3 @ W3[:, :-1]) * (h2 > 0)
    dW2 = np.concatenate([g2.T @ h1, g2.sum(0)[:, None]], axis=1)
    g1 = (g2 @ W2[:, :-1]) * (h1 > 0)
    dW1 = np.concatenate([g1.T @ X, g1.sum(0)[:, None]], axis=1)
    return np.concatenate([dW1.ravel(), dW2.ravel(), dW3.ravel()])


def stencil_index(sk: Skeleton):
    """Global (D index, N index) of every dof row and its 5 stencil rows."""
    D, N, st = [], [], []
    base = 0
    for i in range(sk.n_domains):
        Di, Ni = sk.block_slices(i)
        nb = neighbours(sk, i)
        D.extend(range(Di.start, Di.stop))
        N.extend(range(Ni.start, Ni.stop))
        st.append(np.concatenate([np.arange(sk.N[i])[:, None], nb], axis=1) + base)
        base += sk.N[i]
    return np.array(D), np.array(N), np.concatenate(st)


def correction(sk: Skeleton, y: np.ndarray, r: np.ndarray, pr: np.ndarray) -> np.ndarray:
    """C r for stencil coefficients y (rows, 80) and one vector r with P r."""
    D, N, st = stencil_index(sk)
    a = (y[:, 0::2] + 1j * y[:, 1::2]).reshape(-1, 5, 2, 4)          # [row, q, s, comp]
    sD = np.stack([r[D[st]], pr[D[st]]], axis=2)                       # [row, q, s]
    sN = np.stack([r[N[st]], pr[N[st]]], axis=2)
    z = np.zeros_like(r, dtype=np.complex128)
    z[D] = np.sum(a[..., 0] * sD + a[..., 1] * sN, axis=(1, 2))
    z[N] = np.sum(a[..., 2] * sD + a[..., 3] * sN, axis=(1, 2))
    return z


def correction_matrix(sk: Skeleton, y: np.ndarray, P: np.ndarray) -> np.ndarray:
    """C as a dense matrix (columns: correction of unit vectors)."""
    n = sk.n_total
    C = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        C[:, j] = correction(sk, y, e, P[:, j])
    return C


def coefficient_grad(sk: Skeleton, gz: np.ndarray, r: np.ndarray, pr: np.ndarray) -> np.ndarray:
    """dL/dy (rows, 80) of one vector from g = dL/dRe z + i dL/dIm z (n_total):
    the (re, im) parts of g conj(source) per coefficient."""
    D, N, st = stencil_index(sk)
    sD = np.stack([r[D[st]], pr[D[st]]], axis=2)
    sN = np.stack([r[N[st]], pr[N[st]]], axis=2)
    gD, gN = gz[D][:, None, None], gz[N][:, None, None]
    comp = np.stack([gD * np.conj(sD), gD * np.conj(sN), gN * np.conj(sD), gN * np.conj(sN)], axis=3)
    out = np.zeros((len(D), N_OUT))
    out[:, 0::2] = comp.real.reshape(len(D), -1)
    out[:, 1::2] = comp.imag.reshape(len(D), -1)
    return out


def stencil_adjoint(sk: Skeleton, y: np.ndarray, w: np.ndarray):
    """(C_r^H w, C_P^H w) with C r = C_r r + C_P (P r): every stencil entry of
    row m scattered back to its source dof, the 2 x 2 coupling conjugate-transposed."""
    D, N, st = stencil_index(sk)
    a = (y[:, 0::2] + 1j * y[:, 1::2]).reshape(-1, 5, 2, 4)
    out = []
    for s in range(2):
        o = np.zeros_like(w, dtype=np.complex128)
        wD, wN = w[D][:, None], w[N][:, None]
        np.add.at(o, D[st], np.conj(a[:, :, s, 0]) * wD + np.conj(a[:, :, s, 2]) * wN)
        np.add.at(o, N[st], np.conj(a[:, :, s, 1]) * wD + np.conj(a[:, :, s, 3]) * wN)
        out.append(o)
    return out[0], out[1]


def apply_corrected(sk, M, P, y, e):
    """M (P + C) e."""
    pe = P @ e
    return M @ (pe + correction(sk, y, e, pe))


def power_loss(sk, M, P, y, Z, c0, K):
    """Mean over the rows z of Z of ||E^K z||^2 / ||z||^2, E = I - M (P + C) / c0."""
    tot = 0.0
    for z in Z:
        e = np.array(z, dtype=np.complex128)
        for _ in range(K):
            e = e - apply_corrected(sk, M, P, y, e) / c0
        tot += np.sum(np.abs(e) ** 2) / np.sum(np.abs(z) ** 2)
    return tot / len(Z)


def power_loss_grad(sk, M, P, y, Z, c0, K):
    """(L, dL/dy) of power_loss by reverse accumulation through the K steps:
    a_K = 2 e_K / (||z||^2 |Z|); for j = K-1 .. 0, b = M^H a_{j+1}, dL/dy +=
    coefficient_grad(-b / conj(c0), e_j, P e_j), a_j = a_{j+1} - (P + C)^H b /
    conj(c0) with (P + C)^H b = P^H b + C_r^H b + P^H C_P^H b."""
    G = np.zeros_like(y, dtype=np.float64)
    tot = 0.0
    MH, PH = M.conj().T, P.conj().T
    for z in Z:
        z = np.array(z, dtype=np.complex128)
        es, pes = [z], []
        for _ in range(K):
            pes.append(P @ es[-1])
            es.append(es[-1] - M @ (pes[-1] + correction(sk, y, es[-1], pes[-1])) / c0)
        nz = np.sum(np.abs(z) ** 2)
        tot += np.sum(np.abs(es[K]) ** 2) / nz
        a = 2.0 * es[K] / (nz * len(Z))
        for j in range(K - 1, -1, -1):
            b = MH @ a
            G += coefficient_grad(sk, -b / np.conj(c0), es[j], pes[j])
            cr, cp = stencil_adjoint(sk, y, b)
            a = a - (PH @ b + cr + PH @ cp) / np.conj(c0)
    return tot / len(Z), G
