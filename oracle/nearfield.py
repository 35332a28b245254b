"""Near field by the Stratton-Chu representation, Eq. 8 (oracle side).

Test infrastructure only (imported by tests, never by the product).  For a
point x in Omega_i and the Cauchy data of block i,

    U(x) = H_{k_i}(a)(x) + E_{k_i}(b)(x),   a = gamma_D U,  b = gamma_N U,

with the potentials of Eq. 5:

    H_k a (x) = curl int G(x,y) a(y) dy       = int grad_x G(x,y) x a(y) dy,
    E_k b (x) = i k int G(x,y) b(y) dy - 1/(i k) grad_x int G(x,y) div b(y) dy,
    grad_x G(x,y) = G(x,y) (i k - 1/R) (x - y) / R,   R = |x - y|.

a and b are the RWG fields of block i's D and N coefficients; the N slot of
the unknown holds rho_i gamma_N U, so b uses the coefficients divided by
rho_i.  div of an RWG function is 2 c_a on each of its triangles.  In
Omega_0 the total data give the scattered field (the incident part's
representation vanishes there); at points outside Omega_i the
representation vanishes (the second case of Eq. 8), and block 0's
representation inside the scatterer is -E_inc (the incident field's
interior representation with the opposite normal).  Plain FP64 numpy with
the 6-point triangle rule of the assembly; points must keep about one
triangle diameter from the surface for the rule to resolve G.
"""
from __future__ import annotations

import numpy as np

from .operators import _rwg_data, triangle_points


def representation(ref, x, points, domains):
    """U at points (P, 3) from the solution(s) x (n_total[, nrhs]); domains
    (P,) gives the subdomain of every point.  Returns (P, 3, nrhs) complex."""
    sk = ref.sk
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[:, None]
    points = np.atleast_2d(np.asarray(points, dtype=np.float64))
    domains = np.asarray(domains)
    out = np.zeros((len(points), 3, x.shape[1]), dtype=np.complex128)
    for i in np.unique(domains):
        sel = np.where(domains == i)[0]
        k = complex(ref.k[i])
        rho = complex(ref.rho[i])
        Di, Ni = sk.block_slices(i)
        loc = np.arange(len(sk.tris[i]))
        c, v = _rwg_data(sk, i, loc)                                  # (T,3), (T,3,3)
        Y, W = triangle_points(sk, sk.tris[i])                          # (T,Q,3), (T,Q)
        f = c[:, :, None, None] * (Y[:, None] - v[:, :, None, :])      # (T,3,Q,3)
        dof = sk.dof[i]
        for r in range(x.shape[1]):
            uD = x[Di, r][dof]                                          # (T,3)
            uN = x[Ni, r][dof] / rho
            a = np.einsum("ta,taqn->tqn", uD, f)
            b = np.einsum("ta,taqn->tqn", uN, f)
            divb = np.einsum("ta,ta->t", uN, 2.0 * c)
            for p in sel:
                d = points[p][None, None, :] - Y                       # (T,Q,3)
                R = np.linalg.norm(d, axis=2)
                G = np.exp(1j * k * R) / (4.0 * np.pi * R)
                g = G * (1j * k - 1.0 / R) / R                          # grad G = g d
                gd = g[:, :, None] * d
                H = np.einsum("tq,tqn->n", W, np.cross(gd, a))
                E1 = 1j * k * np.einsum("tq,tq,tqn->n", W, G, b)
                E2 = -(1.0 / (1j * k)) * np.einsum("tq,t,tqn->n", W, divb, gd)
                out[p, :, r] = H + E1 + E2
    return out
