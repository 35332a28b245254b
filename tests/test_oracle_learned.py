"""Oracle of the learned block-OSRC correction (CPU, FP64), pinned
independently: central finite differences of the network loss and of the
training loss with respect to the stencil coefficients, linearity of the
correction, the neighbour relation of RWG dofs and geometric properties of
the features on the split sphere (junction edges on the equator, flat disk)."""
import numpy as np
import pytest

import mtf_inputs as mi
from oracle import learned as Lr
from oracle.mtf import MTFSystem
from oracle.osrc import BlockOSRC
from tests.oracle_helpers import skeleton_of


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    H = 6
    X = rng.standard_normal((29, Lr.N_FEAT))
    T = rng.standard_normal((29, Lr.N_OUT))
    w = rng.uniform(0.5, 2.0, 29)
    theta = rng.standard_normal(Lr.n_params(H)) * 0.3
    L, g = Lr.loss_grad(theta, H, X, T, w)
    h = 1e-6
    for p in rng.choice(len(theta), 60, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += h
        tm[p] -= h
        fd = (Lr.loss_grad(tp, H, X, T, w)[0] - Lr.loss_grad(tm, H, X, T, w)[0]) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1.0, abs(fd)), (p, fd, g[p])


def test_neighbours_are_the_other_edges_of_the_two_triangles():
    sk = skeleton_of(mi.split_sphere(3))
    for i in range(sk.n_domains):
        nb = Lr.neighbours(sk, i)
        assert nb.shape == (sk.N[i], 4)
        for m in range(sk.N[i]):
            assert m not in nb[m]
            for q in nb[m]:
                assert m in nb[q]          # sharing a triangle is symmetric
            tris = np.where((sk.dof[i] == m).any(axis=1))[0]
            assert len(tris) == 2
            assert set(nb[m]) == set(sk.dof[i][tris].ravel()) - {m}


@pytest.fixture(scope="module")
def small_system():
    cfg = mi.config_split_sphere(rings=3, k0=2.0)
    sk = skeleton_of(cfg["mesh"])
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    P = BlockOSRC(sk, ref.k, ref.rho).matrix()
    return sk, ref, ref.matrix(), P


def test_features_geometry(small_system):
    sk, ref, _, _ = small_system
    X = Lr.features(sk, ref.k, ref.rho)
    R = 3
    o = 0
    for i in range(sk.n_domains):
        x = X[o:o + sk.N[i]]
        o += sk.N[i]
        assert np.all(x[:, 2] == (1.0 if i == 0 else 0.0))
        assert np.allclose(x[:, 1], ref.rho[i].real)
        # the 6R equator edges join triangles of two interfaces on every
        # Gamma_i (upper / lower cap on Gamma_0, cap / disk on Gamma_1,2)
        assert int(x[:, 9].sum()) == 6 * R
        assert np.all(x[:, 8] <= 1.0 + 1e-12) and np.all(x[:, 8] >= -1.0 - 1e-12)
        # inside the flat equator disk neighbouring normals are parallel
        if i > 0:
            assert np.sum(np.isclose(x[:, 8], 1.0)) > 0


def test_correction_is_linear_and_zero_for_zero_coefficients(small_system):
    sk, _, _, P = small_system
    rng = np.random.default_rng(2)
    n = sk.n_total
    y = rng.standard_normal((n // 2, Lr.N_OUT))
    r1 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    r2 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    lhs = Lr.correction(sk, y, a * r1 + b * r2, P @ (a * r1 + b * r2))
    rhs = a * Lr.correction(sk, y, r1, P @ r1) + b * Lr.correction(sk, y, r2, P @ r2)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    assert np.all(Lr.correction(sk, 0 * y, r1, P @ r1) == 0)


def test_stencil_adjoint_satisfies_the_inner_product_identity(small_system):
    # <C(r, pr), w> = <r, C_r^H w> + <pr, C_P^H w> for independent r, pr
    sk, _, _, _ = small_system
    rng = np.random.default_rng(4)
    n = sk.n_total
    y = rng.standard_normal((n // 2, Lr.N_OUT))
    r, pr, w = (rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(3))
    cr, cp = Lr.stencil_adjoint(sk, y, w)
    lhs = np.vdot(w, Lr.correction(sk, y, r, pr))
    rhs = np.vdot(cr, r) + np.vdot(cp, pr)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_power_loss_over_the_unit_basis_is_the_frobenius_norm_of_the_propagator(small_system):
    # unit vectors e_k: mean_k ||E^K e_k||^2 = ||E^K||_F^2 / n, E^K by matrix power
    sk, _, M, P = small_system
    rng = np.random.default_rng(5)
    n = sk.n_total
    y = rng.standard_normal((n // 2, Lr.N_OUT)) * 1e-2
    c0, K = -1.5 + 0.1j, 3
    E = np.eye(n) - M @ (P + Lr.correction_matrix(sk, y, P)) / c0
    ref = np.linalg.norm(np.linalg.matrix_power(E, K), "fro") ** 2 / n
    cols = rng.choice(n, 60, replace=False)
    L = Lr.power_loss(sk, M, P, y, np.eye(n)[cols], c0, K)
    EK = np.linalg.matrix_power(E, K)
    assert np.isclose(L, np.mean(np.sum(np.abs(EK[:, cols]) ** 2, 0)), rtol=1e-12)
    Lall = Lr.power_loss(sk, M, P, y, np.eye(n), c0, K)
    assert np.isclose(Lall, ref, rtol=1e-12)


def test_power_loss_gradient_matches_central_differences(small_system):
    sk, _, M, P = small_system
    rng = np.random.default_rng(3)
    n = sk.n_total
    Z = rng.standard_normal((2, n)) + 1j * rng.standard_normal((2, n))
    y = rng.standard_normal((n // 2, Lr.N_OUT)) * 1e-2
    c0, K = -1.6 + 0.05j, 3
    L, g = Lr.power_loss_grad(sk, M, P, y, Z, c0, K)
    assert np.isclose(L, Lr.power_loss(sk, M, P, y, Z, c0, K), rtol=1e-12)
    h = 1e-6
    for _ in range(20):
        row, col = rng.integers(n // 2), rng.integers(Lr.N_OUT)
        yp, ym = y.copy(), y.copy()
        yp[row, col] += h
        ym[row, col] -= h
        fd = (Lr.power_loss(sk, M, P, yp, Z, c0, K) - Lr.power_loss(sk, M, P, ym, Z, c0, K)) / (2 * h)
        assert abs(fd - g[row, col]) <= 1e-5 * max(1.0, abs(fd)), (row, col, fd, g[row, col])
