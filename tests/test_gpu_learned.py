"""Learned block-OSRC correction on the GPU vs the oracle, through the C-ABI.

Parity: features, the network's loss gradient, the stencil, its adjoint, the
adjoint of block-OSRC and the gradient of the power loss (both
parametrisations) against the FP64 oracle with dense M and P on the small
split sphere.  The GPU path computes in FP32, and its adjoint matvec uses
that T and K are complex symmetric (both sides assemble them symmetric to
rounding), hence the norm-wise tolerances 1e-5 (stencil), 1e-4 (operators)
and 3e-4 (gradients through three adjoint steps).  Behaviour: an untrained correction is plain block-OSRC
exactly, training lowers the power loss, and a fitted correction is
measured against plain block-OSRC on plane waves it was not fitted on."""
import numpy as np
import pytest
import torch

import mtf_inputs as mi
from oracle import learned as Lr
from oracle.mtf import MTFSystem
from oracle.osrc import BlockOSRC
from tests.oracle_helpers import skeleton_of

pytestmark = pytest.mark.gpu
H = 256


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import api as A
    return A


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _rand_c64(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.fixture(scope="module")
def small(oracle_cache):
    key = ("learned_small",)
    if key not in oracle_cache:
        cfg = mi.config_split_sphere(rings=3, k0=2.0)
        sk = skeleton_of(cfg["mesh"])
        ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
        oracle_cache[key] = (cfg, sk, ref, ref.matrix(), BlockOSRC(sk, ref.k, ref.rho).matrix())
    return oracle_cache[key]


def _system(api, cfg, **kw):
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    # FP32 T~ so that the block-OSRC parts match the oracle to FP32 accuracy
    opts = dict(precision=1, precond=1, tol=1e-7, restart=200, max_iter=8000, max_refine=8, osrc_half=0)
    opts.update(kw)
    return api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], **opts)


def _random_network(rng, scale_out=0.05):
    th = np.zeros(Lr.n_params(H))
    o = 0
    for k, (a, b) in enumerate(Lr.param_shapes(H)):
        th[o:o + a * b] = rng.standard_normal(a * b) * (0.3 if k < 2 else scale_out)
        o += a * b
    return th.astype(np.float32)


def test_features_match_oracle(api, small):
    cfg, sk, ref, _, _ = small
    sysg = _system(api, cfg)
    sysg.learned_init("network", seed=1)
    X = sysg.learned_features().cpu().numpy().T
    assert rel(X, Lr.features(sk, ref.k, ref.rho)) < 1e-6


def test_network_loss_gradient_matches_oracle(api, small):
    cfg, sk, _, _, _ = small
    sysg = _system(api, cfg)
    sysg.learned_init("network", seed=1)
    rng = np.random.default_rng(0)
    rows = 517                                   # several CTAs and a ragged tail
    X = rng.standard_normal((rows, Lr.N_FEAT)).astype(np.float32)
    T = rng.standard_normal((rows, Lr.N_OUT)).astype(np.float32)
    w = rng.uniform(0.5, 2.0, rows).astype(np.float32)
    th = _random_network(rng, 0.3)
    sysg.learned_params = th
    loss, g = sysg.learned_loss_grad(torch.from_numpy(X.T.copy()).cuda(), torch.from_numpy(T.T.copy()).cuda(),
                                     torch.from_numpy(w).cuda())
    lo, go = Lr.loss_grad(th.astype(np.float64), H, X.astype(np.float64), T.astype(np.float64), w.astype(np.float64))
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    assert rel(g.cpu().numpy(), go) < 1e-4


def _coefficients(sysg, kind, rng, sk, ref):
    """Set random parameters of `kind`; return (params, coefficients (rows, 80), X)."""
    nr = sk.n_total // 2
    if kind == "table":
        y = (rng.standard_normal((nr, Lr.N_OUT)) * 0.05).astype(np.float32)
        sysg.learned_params = y.T.copy().ravel()
        return y, y.astype(np.float64), None
    th = _random_network(rng)
    sysg.learned_params = th
    X = sysg.learned_features().cpu().numpy().T.astype(np.float64)
    return th, Lr.forward(th.astype(np.float64), H, X)[0], X


@pytest.mark.parametrize("kind", ["table", "network"])
def test_stencil_matches_oracle(api, small, kind):
    cfg, sk, ref, _, _ = small
    sysg = _system(api, cfg)
    sysg.learned_init(kind, seed=1)
    rng = np.random.default_rng(1)
    _, y, _ = _coefficients(sysg, kind, rng, sk, ref)
    r = _rand_c64(rng, (3, sk.n_total))
    rt = torch.from_numpy(r).cuda()
    pr = sysg.precond_f32(rt).cpu().numpy().astype(np.complex128)
    z = sysg.learned_apply(rt).cpu().numpy()
    zo = np.stack([pr[c] + Lr.correction(sk, y, r[c].astype(np.complex128), pr[c]) for c in range(3)])
    assert rel(z, zo) < 1e-5


def test_untrained_correction_is_plain_osrc(api, small):
    cfg, sk, _, _, _ = small
    sysg = _system(api, cfg)
    r = torch.from_numpy(_rand_c64(np.random.default_rng(2), (2, sk.n_total))).cuda()
    for kind in ("table", "network"):
        sysg.learned_init(kind, seed=3)
        assert torch.equal(sysg.learned_apply(r), sysg.precond_f32(r))


def test_stencil_adjoint_matches_oracle(api, small):
    cfg, sk, ref, _, _ = small
    sysg = _system(api, cfg)
    sysg.learned_init("table")
    rng = np.random.default_rng(4)
    _, y, _ = _coefficients(sysg, "table", rng, sk, ref)
    w = _rand_c64(rng, (3, sk.n_total))
    cr, cp = sysg.learned_stencil_adjoint(torch.from_numpy(w).cuda())
    ref_r, ref_p = zip(*(Lr.stencil_adjoint(sk, y, w[c].astype(np.complex128)) for c in range(3)))
    assert rel(cr.cpu().numpy(), np.stack(ref_r)) < 1e-5
    assert rel(cp.cpu().numpy(), np.stack(ref_p)) < 1e-5


def test_precond_adjoint_matches_oracle(api, small):
    cfg, sk, _, _, P = small
    sysg = _system(api, cfg)
    w = _rand_c64(np.random.default_rng(5), (5, sk.n_total))
    z = sysg.precond_adjoint_f32(torch.from_numpy(w).cuda()).cpu().numpy()
    zo = (P.conj().T @ w.astype(np.complex128).T).T
    assert rel(z, zo) < 1e-4


@pytest.mark.parametrize("kind", ["table", "network"])
def test_power_loss_gradient_matches_oracle(api, small, kind):
    cfg, sk, ref, M, P = small
    sysg = _system(api, cfg)
    sysg.learned_init(kind, seed=1)
    rng = np.random.default_rng(6)
    th, y, X = _coefficients(sysg, kind, rng, sk, ref)
    Z = _rand_c64(rng, (3, sk.n_total))
    c0, K = -1.6 + 0.05j, 3
    loss, g = sysg.learned_power_grad(torch.from_numpy(Z).cuda(), c0, K)
    lo, G = Lr.power_loss_grad(sk, M, P, y, Z.astype(np.complex128), c0, K)
    assert abs(loss - lo) <= 1e-4 * lo
    if kind == "table":
        go = G.T.ravel()
    else:
        _, acts = Lr.forward(th.astype(np.float64), H, X)
        go = Lr.backward(th.astype(np.float64), H, X, acts, G)
    assert rel(g.cpu().numpy(), go) < 3e-4, rel(g.cpu().numpy(), go)


def test_training_lowers_the_power_loss(api, small):
    cfg, sk, _, _, _ = small
    sysg = _system(api, cfg)
    sysg.learned_init("table")
    c0 = sysg.learned_centre
    Z = torch.from_numpy(_rand_c64(np.random.default_rng(7), (16, sk.n_total))).cuda()
    before, _ = sysg.learned_power_grad(Z, c0, 6)
    l0, l1 = sysg.learned_train(100, lr=3e-3, batch=16, K=6, seed=11)
    after, _ = sysg.learned_power_grad(Z, c0, 6)
    assert np.isfinite(l0) and np.isfinite(l1)
    assert after < 0.5 * before, (before, after)


def test_fitted_correction_against_plain_osrc(api):
    """Fit on two plane waves, validate on them, then solve two others."""
    cfg = mi.config_split_sphere(rings=4, k0=2.0)
    sysg = _system(api, cfg, restart=50)
    sysg.learned_init("table")
    d_val = mi.fibonacci_directions(9)[0:2]
    p_val = mi.orthonormal_polarizations(d_val)[0].astype(np.complex128)
    rep = sysg.learned_fit(d_val, p_val, rounds=4, steps_per_round=150, lr=3e-3, batch=16, K=6, seed=5)
    assert rep["rounds"] == 4 and rep["plain_iterations"] > 0
    assert rep["best_iterations"] <= rep["plain_iterations"]
    assert rep["enabled"] == (1 if rep["best_round"] > 0 else 0)
    d_te = mi.fibonacci_directions(7)[5:7]
    p_te = mi.orthonormal_polarizations(d_te)[0].astype(np.complex128)
    sysg.learned_enable(False)
    x0, st0 = sysg.solve(d_te, p_te)
    sysg.learned_enable(bool(rep["enabled"]))
    x1, st1 = sysg.solve(d_te, p_te)
    assert st0.converged and st1.converged
    # the correction changes the iteration count, not the solution
    assert rel(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-5
    if rep["enabled"]:
        assert st1.iterations <= 1.05 * st0.iterations, (rep, st0.iterations, st1.iterations)


def test_learned_correction_gains_on_held_out_waves(api):
    """The trained correction's gain, measured: on the R = 4 split sphere at
    restart 50 (where restarted GMRES is slowed by the outlying eigenvalues
    of the preconditioned operator that the power loss targets), fit on two
    plane waves and then solve two held-out ones with and without it: at
    least 10% fewer iterations, the same solution to 1e-5."""
    cfg = mi.config_split_sphere(rings=4, k0=2.0)
    sysg = _system(api, cfg, restart=50)
    sysg.learned_init("table")
    d_val = mi.fibonacci_directions(9)[0:2]
    p_val = mi.orthonormal_polarizations(d_val)[0].astype(np.complex128)
    rep = sysg.learned_fit(d_val, p_val, rounds=6, steps_per_round=150, lr=3e-3, batch=16, K=6, seed=5)
    assert rep["enabled"] == 1, rep
    d_te = mi.fibonacci_directions(7)[5:7]
    p_te = mi.orthonormal_polarizations(d_te)[0].astype(np.complex128)
    sysg.learned_enable(False)
    x0, st0 = sysg.solve(d_te, p_te)
    sysg.learned_enable(True)
    x1, st1 = sysg.solve(d_te, p_te)
    assert st0.converged and st1.converged
    assert rel(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-5
    assert st1.iterations <= 0.9 * st0.iterations, (rep, st0.iterations, st1.iterations)
