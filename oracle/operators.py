"""Galerkin operators of the MTF (oracle side, plain FP64 numpy).

Definitions followed (paper, Sec. 2.3 and Sec. 3):

* Helmholtz kernel G_k(x, y) = exp(i k |x-y|) / (4 pi |x-y|)  (Eq. 7).
* Potentials E_k v = i k int G v - 1/(i k) grad int G div v,
  H_k v = curl int G v  (Eq. 7).
* EFIO T_k = {gamma_D E_k}, MFIO K_k = {gamma_D H_k} with gamma_D U = U x n
  (Eqs. 3, 9).
* Galerkin matrices are taken with the self-duality pairing
  <u, v>_x = int u . (n x v)  (Eq. 5) against RWG test functions:
  M_mn = <M psi_n, psi_m>_x  (Sec. 3.2).

Because (a x n) . (n x v) = -a . v for tangential v, the normal cancels in
the EFIO/MFIO pairings and (after integrating the gradient term by parts on
the closed surface Gamma_i)

  T[m, n] = -i k int int G psi_n(y) . psi_m(x) - 1/(i k) int int G div psi_n(y) div psi_m(x)
  K[m, n] = -int int grad_x G(x, y) . (psi_n(y) x psi_m(x))

with grad_x G = G (i k - 1/r) (x - y) / r.  The normal only enters the
identity / transmission Grams and the incident traces.  The overall signs
are those of the definitions above; the test suite checks them against the
Calderon projector identity of Eq. (10) and against the Mie series.
"""
from __future__ import annotations

import numpy as np

from .quadrature import triangle_rule_6, sauter_schwab, ss_map
from .skeleton import Skeleton

FOUR_PI = 4.0 * np.pi


# ----------------------------------------------------------------------------
# quadrature points on triangles
# ----------------------------------------------------------------------------
def triangle_points(sk: Skeleton, tri_ids):
    """Physical points (T, 6, 3) and weights (T, 6) (including 2A) of the
    6-point rule on the given skeleton triangles."""
    s, t, w = triangle_rule_6()
    P = sk.V[sk.F[tri_ids]]  # (T, 3, 3)
    X = (P[:, 0:1, :] + s[None, :, None] * (P[:, 1:2, :] - P[:, 0:1, :])
         + t[None, :, None] * (P[:, 2:3, :] - P[:, 0:1, :]))
    W = 2.0 * sk.area[tri_ids][:, None] * w[None, :]
    return X, W


def _rwg_data(sk: Skeleton, i: int, loc):
    """RWG coefficients c (P,3) and opposite vertices (P,3,3) for local
    triangles ``loc`` of Gamma_i."""
    t = sk.tris[i][loc]
    c = sk.rwg_coeff(i)[loc]
    v = sk.V[sk.F[t]]  # vertex a is opposite local edge a
    return c, v


# ----------------------------------------------------------------------------
# the 3x3 local integrals of one batch of triangle pairs
# ----------------------------------------------------------------------------
def pair_integrals(k, X, Y, W, ca, pa, cb, qb):
    """Local EFIO / MFIO integrals of a batch of triangle pairs.

    X, Y: (P, Q, 3) paired test / trial points; W: (P, Q) weights (including
    both Jacobians); ca, pa: RWG coefficients and opposite vertices of the
    test triangle (P, 3), (P, 3, 3); cb, qb: same for the trial triangle.
    Returns T_loc, K_loc (P, 3, 3) complex, index [a (test), b (trial)].
    """
    R = X - Y
    r = np.linalg.norm(R, axis=-1)
    G = np.exp(1j * k * r) / (FOUR_PI * r)
    gradG = (G * (1j * k - 1.0 / r) / r)[..., None] * R                 # (P,Q,3)
    f = ca[:, :, None, None] * (X[:, None, :, :] - pa[:, :, None, :])   # (P,3,Q,3) test
    g = cb[:, :, None, None] * (Y[:, None, :, :] - qb[:, :, None, :])   # (P,3,Q,3) trial
    divf = 2.0 * ca
    divg = 2.0 * cb
    WG = W * G
    P, Q = W.shape

    def wdot(wt, u, v):
        # sum_q wt[p,q] u[p,a,q,:] . v[p,b,q,:]  as a batched (3 x 3Q)(3Q x 3) product
        uw = (u * wt[:, None, :, None]).reshape(P, 3, 3 * Q)
        return np.matmul(uw, v.reshape(P, 3, 3 * Q).transpose(0, 2, 1))

    T = (-1j * k) * wdot(WG, f.astype(np.complex128), g) \
        - (1.0 / (1j * k)) * (divf[:, :, None] * divg[:, None, :]) * WG.sum(axis=1)[:, None, None]
    # grad G . (g_b x f_a) = f_a . (grad G x g_b)  (cyclic triple product)
    gxg = np.cross(gradG[:, None, :, :], g)                             # (P,3,Q,3)
    K = -wdot(W.astype(np.complex128), f.astype(np.complex128), gxg)
    return T, K


def _shared_vertices(Fa, Fb):
    """Number of common vertex ids of two (P,3) triangle index arrays."""
    return (Fa[:, :, None] == Fb[:, None, :]).sum(axis=(1, 2))


def classify_pairs(sk: Skeleton, i: int):
    """All ordered pairs (tau, sigma) of Gamma_i, split by the number of
    shared vertices: 3 coincident, 2 common edge, 1 common vertex, 0 regular.
    Returns dict kind -> (loc_tau, loc_sigma) arrays of local triangle ids."""
    T = len(sk.tris[i])
    Ft = sk.F[sk.tris[i]]
    a, b = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    a, b = a.ravel(), b.ravel()
    nshared = _shared_vertices(Ft[a], Ft[b])
    names = {3: "coincident", 2: "edge", 1: "vertex", 0: "regular"}
    return {names[c]: (a[nshared == c], b[nshared == c]) for c in (3, 2, 1, 0)}


def ss_vertex_order(Fa, Fb, kind):
    """Vertex orderings (P0, P1, P2) of the test and trial triangles for the
    Sauter-Schwab maps.

    coincident: both keep the stored order.
    edge: shared vertices A, B such that the test triangle's stored cyclic
      order runs A -> B; test = (A, B, C), trial = (A, B, D).
    vertex: shared vertex A; both start at A and keep their cyclic order.
    """
    P = len(Fa)
    oa = np.zeros((P, 3), dtype=np.int64)
    ob = np.zeros((P, 3), dtype=np.int64)
    for p in range(P):
        ta, tb = list(Fa[p]), list(Fb[p])
        if kind == "coincident":
            oa[p], ob[p] = ta, tb
        elif kind == "edge":
            for s in range(3):
                A, B = ta[s], ta[(s + 1) % 3]
                if A in tb and B in tb:
                    C = ta[(s + 2) % 3]
                    D = [v for v in tb if v != A and v != B][0]
                    oa[p], ob[p] = (A, B, C), (A, B, D)
                    break
        else:
            A = [v for v in ta if v in tb][0]
            sa, sb = ta.index(A), tb.index(A)
            oa[p] = (ta[sa], ta[(sa + 1) % 3], ta[(sa + 2) % 3])
            ob[p] = (tb[sb], tb[(sb + 1) % 3], tb[(sb + 2) % 3])
    return oa, ob


def _scatter(Mat, rows, cols, loc):
    """Add local (P,3,3) blocks into Mat at (rows[p,a], cols[p,b])."""
    R = np.broadcast_to(rows[:, :, None], loc.shape)
    C = np.broadcast_to(cols[:, None, :], loc.shape)
    np.add.at(Mat, (R.ravel(), C.ravel()), loc.ravel())


def assemble_block(sk: Skeleton, i: int, k: complex, n_ss: int = 4, chunk: int = 9216,
                   pairs=None):
    """Dense EFIO and MFIO Galerkin matrices T_i, K_i (N_i x N_i) at wavenumber k.

    Regular pairs use the 6x6 tensor rule; singular pairs the Sauter-Schwab
    rules with n_ss Gauss points per coordinate.  ``pairs`` (optional)
    restricts to a dict kind -> (loc_tau, loc_sigma).

    The EFIO and MFIO Galerkin forms are symmetric in test and trial function
    (G(x, y) = G(y, x); for the MFIO the swap changes the sign of both grad G
    and the cross product).  An edge- or vertex-adjacent pair is therefore
    integrated with the lower-indexed triangle as the test triangle, and the
    pair with the roles swapped takes the transposed local block, so that
    both orderings of an adjacent pair come from one Sauter-Schwab rule.
    """
    N = sk.N[i]
    Tm = np.zeros((N, N), dtype=np.complex128)
    Km = np.zeros((N, N), dtype=np.complex128)
    if pairs is None:
        pairs = classify_pairs(sk, i)
    dof = sk.dof[i]
    Xq, Wq = triangle_points(sk, sk.tris[i])
    for kind, (la, lb) in pairs.items():
        # batch size: about ``chunk`` point pairs per numpy call
        npts = 36 if kind == "regular" else len(sauter_schwab(kind, n_ss)[2])
        step = max(1, chunk // npts)
        for s in range(0, len(la), step):
            a0 = la[s:s + step]
            b0 = lb[s:s + len(a0)]
            # adjacent pairs with tau > sigma: integrate (sigma, tau), transpose below
            flip = (a0 > b0) if kind in ("edge", "vertex") else np.zeros(len(a0), dtype=bool)
            a = np.where(flip, b0, a0)
            b = np.where(flip, a0, b0)
            ca, pa = _rwg_data(sk, i, a)
            cb, qb = _rwg_data(sk, i, b)
            if kind == "regular":
                X = np.repeat(Xq[a], 6, axis=1)             # p slow
                Y = np.tile(Xq[b], (1, 6, 1))               # q fast
                W = (Wq[a][:, :, None] * Wq[b][:, None, :]).reshape(len(a), 36)
            else:
                xh, yh, w = sauter_schwab(kind, n_ss)
                Fa = sk.F[sk.tris[i][a]]
                Fb = sk.F[sk.tris[i][b]]
                oa, ob = ss_vertex_order(Fa, Fb, kind)
                X = ss_map(sk.V[oa], xh)
                Y = ss_map(sk.V[ob], yh)
                area_a = sk.area[sk.tris[i][a]]
                area_b = sk.area[sk.tris[i][b]]
                W = (4.0 * area_a * area_b)[:, None] * w[None, :]
            Tl, Kl = pair_integrals(k, X, Y, W, ca, pa, cb, qb)
            Tl = np.where(flip[:, None, None], np.swapaxes(Tl, 1, 2), Tl)
            Kl = np.where(flip[:, None, None], np.swapaxes(Kl, 1, 2), Kl)
            _scatter(Tm, dof[a0], dof[b0], Tl)
            _scatter(Km, dof[a0], dof[b0], Kl)
    return Tm, Km


def block_entries(sk: Skeleton, i: int, k: complex, rows, cols, n_ss: int = 4):
    """Selected entries T_i[rows, cols], K_i[rows, cols] (1-D arrays), each
    summed over the (at most 4) triangle pairs supporting dofs (m, n)."""
    dof = sk.dof[i]
    supp = [[] for _ in range(sk.N[i])]
    for tl in range(len(sk.tris[i])):
        for a in range(3):
            supp[dof[tl, a]].append(tl)
    Ft = sk.F[sk.tris[i]]
    Tout = np.zeros(len(rows), dtype=np.complex128)
    Kout = np.zeros(len(rows), dtype=np.complex128)
    for q, (m, n) in enumerate(zip(rows, cols)):
        pa = np.array([t for t in supp[m] for _ in supp[n]])
        pb = np.array([t for _ in supp[m] for t in supp[n]])
        nsh = _shared_vertices(Ft[pa], Ft[pb])
        names = {3: "coincident", 2: "edge", 1: "vertex", 0: "regular"}
        pairs = {names[c]: (pa[nsh == c], pb[nsh == c]) for c in (3, 2, 1, 0) if np.any(nsh == c)}
        Tm, Km = assemble_block(sk, i, k, n_ss=n_ss, pairs=pairs)
        Tout[q], Kout[q] = Tm[m, n], Km[m, n]
    return Tout, Kout


# ----------------------------------------------------------------------------
# sparse operators: identity and transmission Grams, L2 mass
# ----------------------------------------------------------------------------
def identity_gram(sk: Skeleton, i: int):
    """Id_i[m, n] = <psi_n, psi_m>_{x,i} = int_{Gamma_i} psi_n . (n_i x psi_m)
    (Eq. 5), dense N_i x N_i."""
    N = sk.N[i]
    Id = np.zeros((N, N))
    loc = np.arange(len(sk.tris[i]))
    c, v = _rwg_data(sk, i, loc)
    X, W = triangle_points(sk, sk.tris[i])
    n = sk.outward_normal(i)
    f = c[:, :, None, None] * (X[:, None, :, :] - v[:, :, None, :])   # (T,3,Q,3)
    nxf = np.cross(n[:, None, None, :], f)
    loc3 = np.einsum("tq,tbqn,taqn->tab", W, f, nxf)   # [a test, b trial]
    _scatter(Id, sk.dof[i], sk.dof[i], loc3)
    return Id


def mass_matrix(sk: Skeleton, i: int):
    """L2 Gram int psi_m . psi_n on Gamma_i."""
    N = sk.N[i]
    Mm = np.zeros((N, N))
    loc = np.arange(len(sk.tris[i]))
    c, v = _rwg_data(sk, i, loc)
    X, W = triangle_points(sk, sk.tris[i])
    f = c[:, :, None, None] * (X[:, None, :, :] - v[:, :, None, :])
    _scatter(Mm, sk.dof[i], sk.dof[i], np.einsum("tq,taqn,tbqn->tab", W, f, f))
    return Mm


def transmission_gram(sk: Skeleton, i: int, j: int):
    """G^{ij}[m, n] = <I~^{ji} phi_n, psi_m>_{x,i} = int_{Gamma_ij} phi_n . (n_i x psi_m),
    phi_n in RWG_j, psi_m in RWG_i (Eqs. 11, 12 and Eq. 18); dense N_i x N_j.

    Block row i of the MTF system receives G^{ij} u_j in both trace slots
    (Eq. 13, Remark 2: the same sign for the electric and magnetic traces)."""
    Gm = np.zeros((sk.N[i], sk.N[j]))
    if j not in sk.Lambda[i]:
        return Gm
    lo, hi = min(i, j), max(i, j)
    tris = np.where((sk.L[:, 0] == lo) & (sk.L[:, 1] == hi))[0]
    pos_i = {t: p for p, t in enumerate(sk.tris[i])}
    pos_j = {t: p for p, t in enumerate(sk.tris[j])}
    li = np.array([pos_i[t] for t in tris])
    lj = np.array([pos_j[t] for t in tris])
    ci = sk.rwg_coeff(i)[li]
    cj = sk.rwg_coeff(j)[lj]
    v = sk.V[sk.F[tris]]
    X, W = triangle_points(sk, tris)
    ni = sk.outward_normal(i)[li]
    psi = ci[:, :, None, None] * (X[:, None] - v[:, :, None, :])   # RWG_i (test)
    phi = cj[:, :, None, None] * (X[:, None] - v[:, :, None, :])   # RWG_j (trial)
    nxpsi = np.cross(ni[:, None, None, :], psi)
    loc3 = np.einsum("tq,tbqn,taqn->tab", W, phi, nxpsi)
    _scatter(Gm, sk.dof[i][li], sk.dof[j][lj], loc3)
    return Gm


# ----------------------------------------------------------------------------
# incident data and traces
# ----------------------------------------------------------------------------
def paired_trace(sk: Skeleton, i: int, field_D, field_N):
    """(<gamma_D U, psi_m>_{x,i}, <gamma_N U, psi_m>_{x,i}) for a field given by
    callables field_D(x) = U(x) and field_N(x) = curl U(x) / (i k), evaluated
    with the 6-point rule (gamma_D U = U x n_i, gamma_N U = (curl U / (ik)) x n_i,
    Eq. 3)."""
    loc = np.arange(len(sk.tris[i]))
    c, v = _rwg_data(sk, i, loc)
    X, W = triangle_points(sk, sk.tris[i])
    n = sk.outward_normal(i)[:, None, :]
    f = c[:, :, None, None] * (X[:, None] - v[:, :, None, :])     # (T,3,Q,3)
    nxf = np.cross(n[:, None], f)
    out = []
    for fld in (field_D, field_N):
        U = fld(X)                                                 # (T,Q,3)
        gU = np.cross(U, np.broadcast_to(n, U.shape))
        loc3 = np.einsum("tq,tqn,taqn->ta", W, gU, nxf)
        b = np.zeros(sk.N[i], dtype=np.complex128)
        np.add.at(b, sk.dof[i].ravel(), loc3.ravel())
        out.append(b)
    return out[0], out[1]


def plane_wave(k, d, p):
    """E = p exp(i k d.x) (Eq. 22) and curl E / (i k) = (d x p) exp(i k d.x)."""
    d = np.asarray(d, dtype=np.float64)
    p = np.asarray(p, dtype=np.complex128)
    dxp = np.cross(d, p)

    def E(X):
        return p * np.exp(1j * k * (X @ d))[..., None]

    def N(X):
        return dxp * np.exp(1j * k * (X @ d))[..., None]
    return E, N


def incident_data(sk: Skeleton, k0, d, p):
    """u_0^inc tested on RWG_0: (<gamma_D,0 E_inc, psi_m>_x, <gamma_N,0 E_inc, psi_m>_x)
    (Eq. 14 and Eq. 22)."""
    E, N = plane_wave(k0, d, p)
    return paired_trace(sk, 0, E, N)


def l2_trace_projection(sk: Skeleton, i: int, field_D, field_N):
    """RWG_i coefficients of the L2 projections of gamma_D U and gamma_N U
    (mass-matrix solve), for building discrete Cauchy data of a known field."""
    loc = np.arange(len(sk.tris[i]))
    c, v = _rwg_data(sk, i, loc)
    X, W = triangle_points(sk, sk.tris[i])
    n = sk.outward_normal(i)[:, None, :]
    f = c[:, :, None, None] * (X[:, None] - v[:, :, None, :])
    Mm = mass_matrix(sk, i)
    out = []
    for fld in (field_D, field_N):
        U = fld(X)
        gU = np.cross(U, np.broadcast_to(n, U.shape))
        loc3 = np.einsum("tq,tqn,taqn->ta", W, gU, f)
        b = np.zeros(sk.N[i], dtype=np.complex128)
        np.add.at(b, sk.dof[i].ravel(), loc3.ravel())
        out.append(np.linalg.solve(Mm, b))
    return out[0], out[1]


def block_rows(sk: Skeleton, i: int, k: complex, rows, n_ss: int = 4):
    """Full rows T_i[rows, :], K_i[rows, :]: assembles every pair whose test
    triangle supports one of the rows (the only pairs that touch them)."""
    rows = np.asarray(rows)
    dof = sk.dof[i]
    tau = np.unique(np.where(np.isin(dof, rows).any(axis=1))[0])
    T = len(sk.tris[i])
    a = np.repeat(tau, T)
    b = np.tile(np.arange(T), len(tau))
    Ft = sk.F[sk.tris[i]]
    nsh = _shared_vertices(Ft[a], Ft[b])
    names = {3: "coincident", 2: "edge", 1: "vertex", 0: "regular"}
    pairs = {names[c]: (a[nsh == c], b[nsh == c]) for c in (3, 2, 1, 0) if np.any(nsh == c)}
    Tm, Km = assemble_block(sk, i, k, n_ss=n_ss, pairs=pairs)
    return Tm[rows], Km[rows]
