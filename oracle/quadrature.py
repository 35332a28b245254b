"""Quadrature rules, generated from their defining equations (oracle side).

The paper assembles with Bempp-cl's defaults (Sec. 5.1) without stating the
rules.  Reading taken (shared with the CUDA library, which generates its own
copy of the same rules independently):

* regular (vertex-disjoint) triangle pairs: tensor product of the fully
  symmetric 6-point triangle rule of polynomial degree 4 (two orbits of
  three points), obtained here by Newton's method on its moment equations;
* singular pairs (coincident, common edge, common vertex): the Sauter-Schwab
  transformations (Sauter & Schwab, Boundary Element Methods, 2011, Sec. 5.2)
  to the unit 4-cube with an n-point Gauss-Legendre rule per coordinate.

Reference triangle of the regular rule: {(s, t): s, t >= 0, s + t <= 1}
(area 1/2), point x = v0 + s (v1 - v0) + t (v2 - v0).
Reference triangle of the singular rules: K = {(x1, x2): 0 <= x2 <= x1 <= 1}
(area 1/2), point x = P0 + x1 (P1 - P0) + x2 (P2 - P1).
"""
from __future__ import annotations

import functools
import math

import numpy as np


@functools.lru_cache(maxsize=None)
def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1].

    Nodes are the roots of P_n found by Newton's method with the three-term
    recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; weights are
    2 / ((1 - x^2) P_n'(x)^2) on [-1, 1], halved for [0, 1].
    """
    x = np.cos(np.pi * (np.arange(1, n + 1) - 0.25) / (n + 0.5))
    for _ in range(100):
        p0, p1 = np.ones_like(x), x.copy()
        for k in range(1, n):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0, p1 = np.ones_like(x), x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return (x[order] + 1.0) / 2.0, w[order] / 2.0


@functools.lru_cache(maxsize=None)
def triangle_rule_6():
    """Fully symmetric 6-point rule of degree 4 on the reference triangle.

    Points are the S3-orbits of the barycentric triples (a, a, 1-2a) and
    (b, b, 1-2b) with weights wa, wb.  A symmetric rule is exact up to
    degree 4 iff it integrates the invariants 1, e2, e3 and e2^2 exactly
    (e2 = l0 l1 + l0 l2 + l1 l2, e3 = l0 l1 l2), whose integrals over the
    reference triangle follow from int l0^i l1^j l2^k = i! j! k! / (i+j+k+2)!:
    1/2, 1/8, 1/120, 1/30.  Those four equations are solved by Newton's
    method.  Returns (s, t, w) arrays with the barycentric order
    (l0, l1, l2) = (1-2a, a, a), (a, 1-2a, a), (a, a, 1-2a) for each orbit,
    s = l1, t = l2, sum(w) = 1/2.
    """
    target = np.array([1 / 2, 1 / 8, 1 / 120, 1 / 30])

    def inv(a):
        e2 = 2 * a - 3 * a * a
        e3 = a * a * (1 - 2 * a)
        return np.array([1.0, e2, e3, e2 * e2])

    def F(z):
        a, b, wa, wb = z
        return 3 * wa * inv(a) + 3 * wb * inv(b) - target

    z = np.array([0.44, 0.09, 0.11, 0.055])
    for _ in range(60):
        f = F(z)
        J = np.empty((4, 4))
        for c in range(4):
            dz = np.zeros(4)
            dz[c] = 1e-7
            J[:, c] = (F(z + dz) - F(z - dz)) / 2e-7
        step = np.linalg.solve(J, f)
        z = z - step
        if np.max(np.abs(step)) < 1e-15:
            break
    a, b, wa, wb = z
    s, t, w = [], [], []
    for (c, wc) in ((a, wa), (b, wb)):
        for lam in ((1 - 2 * c, c, c), (c, 1 - 2 * c, c), (c, c, 1 - 2 * c)):
            s.append(lam[1])
            t.append(lam[2])
            w.append(wc)
    return np.array(s), np.array(t), np.array(w)


@functools.lru_cache(maxsize=None)
def sauter_schwab(kind: str, n: int):
    """Sauter-Schwab rule for a singular triangle pair on K x K.

    Returns (xh, yh, w): xh, yh (npts, 2) reference coordinates in
    K = {0 <= x2 <= x1 <= 1} of the test and trial points, w (npts,) the
    weights including the Jacobian of the transformation from [0,1]^4, so that
    int_K int_K f(x, y) dy dx ~= sum w f(xh, yh).

    kind = "coincident": same triangle, same parametrisation (6 regions,
    Jacobian xi^3 eta1^2 eta2).
    kind = "edge": the common edge is P0->P1 (x2 = 0) in both parametrisations
    (5 regions, Jacobians xi^3 eta1^2 and xi^3 eta1^2 eta2).
    kind = "vertex": the common vertex is P0 (origin) in both (2 regions,
    Jacobian xi^3 eta2).
    Region order and point order (xi slowest, eta3 fastest) are part of the
    rule's definition, so that both implementations sum identically.
    """
    g, gw = gauss_legendre(n)
    xi, e1, e2, e3 = np.meshgrid(g, g, g, g, indexing="ij")
    W4 = np.einsum("a,b,c,d->abcd", gw, gw, gw, gw)
    xi, e1, e2, e3, W4 = (a.ravel() for a in (xi, e1, e2, e3, W4))
    regions = []
    if kind == "coincident":
        J = xi ** 3 * e1 ** 2 * e2
        regions = [
            ((xi, xi * (1 - e1 + e1 * e2)), (xi * (1 - e1 * e2 * e3), xi * (1 - e1))),
            ((xi * (1 - e1 * e2 * e3), xi * (1 - e1)), (xi, xi * (1 - e1 + e1 * e2))),
            ((xi, xi * e1 * (1 - e2 + e2 * e3)), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
            ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * (1 - e2 + e2 * e3))),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * (1 - e2))),
            ((xi, xi * e1 * (1 - e2)), (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3))),
        ]
        jac = [J] * 6
    elif kind == "edge":
        J1 = xi ** 3 * e1 ** 2
        J2 = xi ** 3 * e1 ** 2 * e2
        regions = [
            ((xi, xi * e1 * e3), (xi * (1 - e1 * e2), xi * e1 * (1 - e2))),
            ((xi, xi * e1), (xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3))),
            ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * e2 * e3)),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), (xi, xi * e1)),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * e2)),
        ]
        jac = [J1, J2, J2, J2, J2]
    elif kind == "vertex":
        J = xi ** 3 * e2
        regions = [
            ((xi, xi * e1), (xi * e2, xi * e2 * e3)),
            ((xi * e2, xi * e2 * e3), (xi, xi * e1)),
        ]
        jac = [J, J]
    else:
        raise ValueError(kind)
    xs, ys, ws = [], [], []
    for ((x1, x2), (y1, y2)), J in zip(regions, jac):
        xs.append(np.stack([x1, x2], axis=1))
        ys.append(np.stack([y1, y2], axis=1))
        ws.append(W4 * J)
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ws)


def ss_map(P, xh):
    """Sauter-Schwab parametrisation x = P0 + x1 (P1 - P0) + x2 (P2 - P1).

    P: (..., 3, 3) vertices (P0, P1, P2); xh: (npts, 2).  Returns (..., npts, 3).
    """
    P0, P1, P2 = P[..., 0:1, :], P[..., 1:2, :], P[..., 2:3, :]
    return P0 + xh[:, 0:1] * (P1 - P0) + xh[:, 1:2] * (P2 - P1)


def simplex_monomial_integral(i: int, j: int, k: int) -> float:
    """Exact int over the reference triangle of l0^i l1^j l2^k (area 1/2)."""
    return math.factorial(i) * math.factorial(j) * math.factorial(k) / math.factorial(i + j + k + 2)
