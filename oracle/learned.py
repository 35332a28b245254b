"""Learned correction of the block-OSRC preconditioner (oracle side).

Test infrastructure only (imported by tests, never by the product).  The
paper has no learned part; this is the reading the library implements:

* Preconditioner: z = P r + s g(x(r)), P the block-OSRC operator (Eq. 19),
  s = sqrt(sum |r|^2 / n) the RMS of r over its n complex entries, and g a
  per-dof multilayer perceptron whose 4 outputs are the real and imaginary
  parts of the correction of the D and N slots of that dof.
* Features x of dof m of block i (43 values): the 8 reals
  (r_D, r_N, (P r)_D, (P r)_N) / s at m, the same 8 at its 4 RWG neighbours
  (the other edges of the two triangles of Gamma_i that share edge m,
  ascending local dof index), k_i l_m (wavenumber x edge length), rho_i,
  and 1 for the exterior block (i = 0), else 0.
* Network: x -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3, hidden
  width H; parameters stored as augmented matrices [W | b] row-major, layer
  after layer (W1: H x 44, W2: H x (H+1), W3: 4 x (H+1)).
* Loss of a batch of exact pairs (r, e) with M e = r: the mean over pairs of
  ||P r + s g - e||^2 / ||e||^2 = sum over rows of w_row |g(x) - t|^2 with
  t = (e - P r) / s and w_row = s^2 / (||e||^2 * pairs).

Everything here is plain FP64 numpy written from these definitions.
"""
from __future__ import annotations

import numpy as np

from .skeleton import Skeleton

N_FEAT = 43
N_OUT = 4


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


def features(sk: Skeleton, k, rho, r: np.ndarray, pr: np.ndarray) -> np.ndarray:
    """Features (rows, 43) of one vector r (n_total complex) and P r; rows in the
    global dof order (block by block, dof by dof)."""
    n = sk.n_total
    s = np.sqrt(np.sum(np.abs(r) ** 2) / n)
    s = s if s > 0 else 1.0
    rows = []
    for i in range(sk.n_domains):
        Di, Ni = sk.block_slices(i)
        rD, rN, pD, pN = r[Di] / s, r[Ni] / s, pr[Di] / s, pr[Ni] / s
        loc = np.stack([rD.real, rD.imag, rN.real, rN.imag, pD.real, pD.imag, pN.real, pN.imag], axis=1)
        nb = neighbours(sk, i)
        E = sk.edges[i]
        le = np.linalg.norm(sk.V[E[:, 1]] - sk.V[E[:, 0]], axis=1)
        x = np.zeros((sk.N[i], N_FEAT))
        x[:, 0:8] = loc
        for q in range(4):
            x[:, 8 + 8 * q: 16 + 8 * q] = loc[nb[:, q]]
        x[:, 40] = np.real(k[i]) * le
        x[:, 41] = np.real(rho[i])
        x[:, 42] = 1.0 if i == 0 else 0.0
        rows.append(x)
    return np.concatenate(rows, axis=0), s


def correction_rows_to_vector(sk: Skeleton, y: np.ndarray) -> np.ndarray:
    """Per-row outputs (rows, 4) -> complex vector (n_total) in the [D, N] block layout."""
    z = np.zeros(sk.n_total, dtype=np.complex128)
    o = 0
    for i in range(sk.n_domains):
        Di, Ni = sk.block_slices(i)
        yi = y[o:o + sk.N[i]]
        z[Di] = yi[:, 0] + 1j * yi[:, 1]
        z[Ni] = yi[:, 2] + 1j * yi[:, 3]
        o += sk.N[i]
    return z


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
    """Outputs (rows, 4) and the activations needed by backward."""
    W1, W2, W3 = unpack(theta, H)
    a1 = X @ W1[:, :-1].T + W1[:, -1]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2[:, :-1].T + W2[:, -1]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3[:, :-1].T + W3[:, -1]
    return y, (h1, h2)


def loss_grad(theta, H, X, T, w):
    """L = sum_rows w_row |y - t|^2 and dL/dtheta (same layout as theta)."""
    W1, W2, W3 = unpack(theta, H)
    y, (h1, h2) = forward(theta, H, X)
    d = y - T
    L = float(np.sum(w[:, None] * d * d))
    g3 = 2.0 * w[:, None] * d                         # dL/dy
    dW3 = np.concatenate([g3.T @ h2, g3.sum(0)[:, None]], axis=1)
    g2 = (g3 @ W3[:, :-1]) * (h2 > 0)
    dW2 = np.concatenate([g2.T @ h1, g2.sum(0)[:, None]], axis=1)
    g1 = (g2 @ W2[:, :-1]) * (h1 > 0)
    dW1 = np.concatenate([g1.T @ X, g1.sum(0)[:, None]], axis=1)
    return L, np.concatenate([dW1.ravel(), dW2.ravel(), dW3.ravel()])


def pair_rows(sk: Skeleton, k, rho, r, pr, e, n_pairs: int):
    """Features, targets and row weights of one exact pair (M e = r)."""
    X, s = features(sk, k, rho, r, pr)
    t = (e - pr) / s
    T = np.zeros((X.shape[0], N_OUT))
    o = 0
    for i in range(sk.n_domains):
        Di, Ni = sk.block_slices(i)
        T[o:o + sk.N[i], 0] = t[Di].real
        T[o:o + sk.N[i], 1] = t[Di].imag
        T[o:o + sk.N[i], 2] = t[Ni].real
        T[o:o + sk.N[i], 3] = t[Ni].imag
        o += sk.N[i]
    w = np.full(X.shape[0], s * s / (np.sum(np.abs(e) ** 2) * n_pairs))
    return X, T, w
