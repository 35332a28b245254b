"""Independent nested quadrature of singular triangle-pair integrals.

Test-only pin for the Sauter-Schwab rules (no Sauter-Schwab map is used
here).  The pair integral int_tau int_sigma F(x, y) dy dx is computed as an
outer rule over tau of the inner integral over sigma, and the inner integral
is taken in polar-type coordinates about the projection x' of x onto the
plane of sigma: sigma is the signed union of the three triangles
(x', s_k, s_k+1), each parametrised by y = x' + s (u + t (v - u)),
dy = s J ds dt, which cancels the 1/|x - y| singularity.  Both coordinates
use composite Gauss-Legendre rules graded towards the singular points
(s -> 0, and t -> the foot of the perpendicular from x' to the edge line).
The outer rule over tau is graded towards the part of tau's boundary where
the inner integral loses smoothness (the common edge, common vertex, or the
whole boundary for coincident triangles).
"""
from __future__ import annotations

import numpy as np

from .quadrature import gauss_legendre

FOUR_PI = 4.0 * np.pi


def _graded(n, q):
    """Nodes/weights on [0, 1] of z -> z^q applied to an n-point Gauss rule."""
    z, w = gauss_legendre(n)
    return z ** q, w * q * z ** (q - 1)


def inner_integrals(x, S, k, cb, qb, ns=20, nt=20, q=4):
    """For each x (B, 3): A[b] = int_sigma G g_b, D[b] = int_sigma G div g_b,
    H[b] = int_sigma grad_x G x g_b, with g_b = cb[b] (y - qb[b])."""
    B = len(x)
    nrm = np.cross(S[1] - S[0], S[2] - S[0])
    nrm /= np.linalg.norm(nrm)
    h = (x - S[0]) @ nrm
    xp = x - h[:, None] * nrm
    sz, sw = _graded(ns, q)
    tz, tw = _graded(nt, q)
    A = np.zeros((B, 3, 3), dtype=np.complex128)
    D = np.zeros((B, 3), dtype=np.complex128)
    H = np.zeros((B, 3, 3), dtype=np.complex128)
    for kk in range(3):
        a, b = S[kk], S[(kk + 1) % 3]
        u = a - xp
        v = b - xp
        J = np.cross(u, v) @ nrm                                    # (B,)
        e = b - a
        tstar = np.clip(((xp - a) @ e) / (e @ e), 0.0, 1.0)         # (B,)
        # t nodes: [0, t*] graded towards t*, [t*, 1] graded towards t*
        tl = tstar[:, None] * (1.0 - tz[None, :])
        wl = tstar[:, None] * tw[None, :]
        tr = tstar[:, None] + (1.0 - tstar[:, None]) * tz[None, :]
        wr = (1.0 - tstar[:, None]) * tw[None, :]
        t = np.concatenate([tl, tr], axis=1)                        # (B, 2nt)
        wt = np.concatenate([wl, wr], axis=1)
        wdir = u[:, None, :] + t[..., None] * (v - u)[:, None, :]   # (B, T, 3)
        y = xp[:, None, None, :] + sz[None, None, :, None] * wdir[:, :, None, :]  # (B,T,S,3)
        wgt = (J[:, None, None] * wt[:, :, None] * sw[None, None, :] * sz[None, None, :])
        # x - y formed from relative quantities (h n - s w), not by
        # subtracting nearly equal points
        R = h[:, None, None, None] * nrm - sz[None, None, :, None] * wdir[:, :, None, :]
        r = np.linalg.norm(R, axis=-1)
        G = np.exp(1j * k * r) / (FOUR_PI * r)
        gradG = (G * (1j * k - 1.0 / r) / r)[..., None] * R
        for bb in range(3):
            g = cb[bb] * (y - qb[bb])
            A[:, bb, :] += np.einsum("bts,btsn->bn", wgt * G, g)
            D[:, bb] += 2.0 * cb[bb] * np.einsum("bts->b", wgt * G)
            H[:, bb, :] += np.einsum("bts,btsn->bn", wgt, np.cross(gradG, g))
    return A, D, H


def outer_points(P, kind, n=16, q=4):
    """Graded outer rule on triangle P (3, 3) (the test triangle).

    kind = 'edge': graded towards the edge P0-P1; 'vertex': towards P0;
    'coincident': three sub-triangles from the centroid, each graded towards
    its outer edge.  Returns points (B, 3) and weights (B,)."""
    if kind == "coincident":
        c = P.mean(axis=0)
        pts, wts = [], []
        for kk in range(3):
            sub = np.array([P[kk], P[(kk + 1) % 3], c])
            p, w = outer_points(sub, "edge", n, q)
            pts.append(p)
            wts.append(w)
        return np.concatenate(pts), np.concatenate(wts)
    # parametrise x = P0 + u (P1 - P0) + u v (P2 - P1) on u, v in [0, 1]
    # (Jacobian 2A u); the edge P0-P1 is v = 0, the vertex P0 is u = 0.
    area2 = np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    if kind == "edge":
        uz, uw = gauss_legendre(n)
        uz = np.concatenate([uz / 2, 0.5 + uz / 2])  # composite, two panels
        uw = np.concatenate([uw / 2, uw / 2])
        vz, vw = _graded(n, q)
    else:
        uz, uw = _graded(n, q)
        vz, vw = gauss_legendre(n)
    U, Vv = np.meshgrid(uz, vz, indexing="ij")
    W = np.outer(uw, vw) * U * area2
    X = P[0] + U[..., None] * (P[1] - P[0]) + (U * Vv)[..., None] * (P[2] - P[1])
    return X.reshape(-1, 3), W.ravel()


def brute_pair(k, Ptau, Psig, ca, pa, cb, qb, kind, n_outer=16, n_inner=20):
    """3x3 local EFIO / MFIO integrals of the pair (tau, sigma) by nested
    quadrature; same definitions as oracle.operators.pair_integrals.
    For kind = 'edge' Ptau must list the common edge first (P0, P1); for
    'vertex' the common vertex first."""
    X, W = outer_points(Ptau, kind, n_outer)
    T = np.zeros((3, 3), dtype=np.complex128)
    K = np.zeros((3, 3), dtype=np.complex128)
    for s0 in range(0, len(X), 256):
        x, w = X[s0:s0 + 256], W[s0:s0 + 256]
        A, D, H = inner_integrals(x, Psig, k, cb, qb, ns=n_inner, nt=n_inner)
        f = ca[None, :, None] * (x[:, None, :] - pa[None, :, :])      # (B,3a,3)
        divf = 2.0 * ca
        T += (-1j * k) * np.einsum("b,ban,bcn->ac", w, f, A) \
            - (1.0 / (1j * k)) * np.einsum("b,a,bc->ac", w, divf, D)
        K += -np.einsum("b,ban,bcn->ac", w, f, H)
    return T, K
