"""Oracle of the learned OSRC correction (CPU, FP64), pinned independently:
central finite differences of its own loss, the vector form of the loss, the
neighbour relation of RWG dofs and the scale invariance of the features."""
import numpy as np
import pytest

import mtf_inputs as mi
from oracle import learned as Lr
from oracle.mtf import MTFSystem
from tests.oracle_helpers import skeleton_of


def _rand_theta(rng, H, scale=0.3):
    return rng.standard_normal(Lr.n_params(H)) * scale


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    H = 6
    X = rng.standard_normal((37, Lr.N_FEAT))
    T = rng.standard_normal((37, Lr.N_OUT))
    w = rng.uniform(0.5, 2.0, 37)
    theta = _rand_theta(rng, H)
    L, g = Lr.loss_grad(theta, H, X, T, w)
    h = 1e-6
    idx = rng.choice(len(theta), 60, replace=False)
    for p in idx:
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
    return sk, ref


def test_features_scale_invariant_and_loss_equals_vector_form(small_system):
    sk, ref = small_system
    rng = np.random.default_rng(1)
    n = sk.n_total
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    pr = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    e = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X1, s1 = Lr.features(sk, ref.k, ref.rho, r, pr)
    X2, s2 = Lr.features(sk, ref.k, ref.rho, 3.7 * r, 3.7 * pr)
    assert np.allclose(X1, X2, rtol=1e-13, atol=1e-13) and np.isclose(s2, 3.7 * s1)
    H = 5
    theta = _rand_theta(rng, H)
    X, T, w = Lr.pair_rows(sk, ref.k, ref.rho, r, pr, e, n_pairs=1)
    L, _ = Lr.loss_grad(theta, H, X, T, w)
    y, _ = Lr.forward(theta, H, X)
    z = pr + s1 * Lr.correction_rows_to_vector(sk, y)
    assert np.isclose(L, np.sum(np.abs(z - e) ** 2) / np.sum(np.abs(e) ** 2), rtol=1e-12)
    # a zero output layer is plain OSRC
    theta0 = theta.copy()
    theta0[-Lr.N_OUT * (H + 1):] = 0.0
    L0, _ = Lr.loss_grad(theta0, H, X, T, w)
    assert np.isclose(L0, np.sum(np.abs(pr - e) ** 2) / np.sum(np.abs(e) ** 2), rtol=1e-12)
