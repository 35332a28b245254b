"""Pins of the quadrature rules against exact integrals (no GPU)."""
import math

import numpy as np
import pytest

from oracle.quadrature import (gauss_legendre, triangle_rule_6, sauter_schwab,
                               simplex_monomial_integral)


@pytest.mark.parametrize("n", [1, 2, 4, 7, 12])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = gauss_legendre(n)
    for j in range(2 * n):
        assert abs(np.sum(w * x ** j) - 1.0 / (j + 1)) < 1e-14
    # not exact at degree 2n (the defect is large enough to see for small n)
    if n <= 7:
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


def test_triangle_rule_6_degree_4():
    s, t, w = triangle_rule_6()
    assert len(w) == 6 and np.all(w > 0) and np.all(s > 0) and np.all(t > 0) and np.all(s + t < 1)
    for a in range(5):
        for b in range(5 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(np.sum(w * s ** a * t ** b) - exact) < 1e-15
    # degree 5 is not integrated exactly
    errs = [abs(np.sum(w * s ** a * t ** (5 - a)) - math.factorial(a) * math.factorial(5 - a) / math.factorial(7))
            for a in range(6)]
    assert max(errs) > 1e-8
    # barycentric monomials
    l0 = 1 - s - t
    assert abs(np.sum(w * l0 * s * t) - simplex_monomial_integral(1, 1, 1)) < 1e-16


def _exact_K(a, b):
    # int over K = {0 <= x2 <= x1 <= 1} of x1^a x2^b
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("kind", ["coincident", "edge", "vertex"])
def test_sauter_schwab_integrates_polynomials_exactly(kind):
    """The transformations must tile K x K exactly once with the right
    Jacobian: polynomials in (x, y) are integrated exactly once n is large."""
    xh, yh, w = sauter_schwab(kind, 8)
    for (a, b, c, d) in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1),
                         (2, 1, 0, 1), (1, 2, 3, 0), (0, 3, 1, 2), (3, 0, 2, 2), (1, 1, 1, 1)]:
        q = np.sum(w * xh[:, 0] ** a * xh[:, 1] ** b * yh[:, 0] ** c * yh[:, 1] ** d)
        ex = _exact_K(a, b) * _exact_K(c, d)
        assert abs(q - ex) < 1e-13 * max(1.0, ex) + 1e-15, (a, b, c, d, q, ex)
    # all points in K
    for P in (xh, yh):
        assert np.all(P[:, 1] <= P[:, 0] + 1e-15) and np.all(P >= 0) and np.all(P <= 1)


def test_sauter_schwab_singularity_location():
    """coincident: x = y on the diagonal only in the xi -> 0 limit of each
    region; edge: the singular set x2 = y2 = 0, x1 = y1 is approached as
    eta1 -> 0; vertex: x = y = 0 only at xi -> 0.  Check that |x - y| scales
    with the collapsing coordinate (which is what cancels 1/r)."""
    for kind in ("coincident", "edge", "vertex"):
        xh, yh, w = sauter_schwab(kind, 3)
        d = np.linalg.norm(xh - yh, axis=1)
        assert np.all(d > 0)
        # the Jacobian-weighted 1/r integrand is bounded: w / r stays finite
        assert np.isfinite(np.max(w / d))
