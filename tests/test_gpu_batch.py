"""Batched solve of independent instances (mtf_solve_batch) and the
operator-apply autotuner (mtf_autotune), through the C-ABI, against the
oracle's LU solution of every instance of the same discrete systems.

Four uneven instances of the batched workload's family (spheres cut by
parallel planes into 4..15 slab subdomains, rotated at random; 1,464 to 2,844
unknowns), 8 plane waves each, solved together:
* FP64 path with block-OSRC: every instance within 1e-10 of its LU solution;
* mixed path with block-OSRC (block FGMRES and tensor-core applies for the
  8 waves): every instance within 1e-5, and the same iterate as a single
  solve of that instance to rounding;
* the mixed path with FP64 refinement residuals (residual_fp64): within 1e-7
  at tol 1e-10, beyond what the FP32-stored operator allows;
* the autotuner times its candidate apply plans, keeps one, and the tuned
  system still matches the oracle (matvec at 1e-5, solve at 1e-5)."""
import numpy as np
import pytest
import torch

import mtf_inputs as mi
from oracle.mtf import MTFSystem
from tests.oracle_helpers import skeleton_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def instances():
    out = []
    for cfg in mi.config_batch_instances(n_inst=4, seed=3, tri_range=(250, 500), nrhs=8):
        sk = skeleton_of(cfg["mesh"])
        ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
        pols = np.array(cfg["pols"], dtype=np.complex128)
        xr = ref.solve_lu(ref.rhs(cfg["dirs"], pols)).T  # (nrhs, n)
        out.append((cfg, sk, ref, xr))
    return out


def _errs(x, xr):
    x = x.cpu().numpy()
    return np.linalg.norm(x - xr, axis=1) / np.linalg.norm(xr, axis=1)


def test_batch_fp64_and_mixed_match_oracle_lu(api, instances):
    meshes = [api.Mesh.from_inputs(cfg["mesh"]) for cfg, _, _, _ in instances]
    dirs = [cfg["dirs"] for cfg, _, _, _ in instances]
    pols = [np.array(cfg["pols"], dtype=np.complex128) for cfg, _, _, _ in instances]
    s64 = [api.System(m, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precond=1, tol=1e-12, restart=1000, max_iter=6000)
           for m, (cfg, _, _, _) in zip(meshes, instances)]
    xs, st = api.solve_batch(s64, dirs, pols, threads=4)
    for x, s, (_, _, _, xr) in zip(xs, st, instances):
        assert s.converged == 1
        assert _errs(x, xr).max() < 1e-10
    s32 = [api.System(m, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8, restart=500,
                      max_iter=6000, max_refine=6) for m, (cfg, _, _, _) in zip(meshes, instances)]
    xs, st = api.solve_batch(s32, dirs, pols)
    for x, s, (_, _, _, xr) in zip(xs, st, instances):
        assert s.converged == 1
        assert _errs(x, xr).max() < 1e-5, _errs(x, xr)
    # a single solve of one instance gives the batch's iterate to rounding
    x0, _ = s32[0].solve(dirs[0], pols[0])
    d = (x0 - xs[0]).abs().max().item() / xs[0].abs().max().item()
    assert d < 1e-9, d
    # residual_fp64: refinement residuals of the FP64 blocks, so the mixed
    # solve converges to the FP64 system's solution, past the FP32 floor
    sdf = [api.System(m, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-10, restart=500,
                      max_iter=8000, max_refine=10, residual_fp64=1) for m, (cfg, _, _, _) in zip(meshes, instances)]
    xs, st = api.solve_batch(sdf, dirs, pols)
    for x, s, (_, _, _, xr) in zip(xs, st, instances):
        assert s.converged == 1
        assert _errs(x, xr).max() < 1e-7, _errs(x, xr)


def test_batch_rejects_a_repeated_system(api, instances):
    cfg = instances[0][0]
    m = api.Mesh.from_inputs(cfg["mesh"])
    s = api.System(m, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1)
    with pytest.raises(api.L.MtfError):
        api.solve_batch([s, s], [cfg["dirs"]] * 2, [cfg["pols"]] * 2)


def test_autotuned_system_matches_oracle(api, instances):
    cfg, sk, ref, xr = instances[0]
    m = api.Mesh.from_inputs(cfg["mesh"])
    s = api.System(m, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8, restart=500,
                   max_iter=6000, max_refine=6)
    report = s.autotune(8, reps=3)
    assert len(report) >= 3 and report[-1].startswith("chosen "), report
    assert any(r.startswith("fma_stream ") for r in report) and any(r.startswith("tc ") for r in report)
    rng = np.random.default_rng(4)
    x = (rng.standard_normal((8, sk.n_total)) + 1j * rng.standard_normal((8, sk.n_total))).astype(np.complex64)
    y = s.matvec_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    yr = np.stack([ref.matvec(xx.astype(np.complex128)) for xx in x])
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < 1e-5
    xt, st = s.solve(cfg["dirs"], np.array(cfg["pols"], dtype=np.complex128))
    assert st.converged == 1
    assert _errs(xt, xr).max() < 1e-5


def test_batch_reports_the_failing_instance_and_finishes_the_others(api, instances):
    """An instance that cannot reach its tolerance within its iteration cap
    makes the batch return MTF_ERR_NOCONV (with raise_on_noconv off), while
    every other instance still runs to its own converged solution."""
    meshes = [api.Mesh.from_inputs(cfg["mesh"]) for cfg, _, _, _ in instances]
    dirs = [cfg["dirs"] for cfg, _, _, _ in instances]
    pols = [np.array(cfg["pols"], dtype=np.complex128) for cfg, _, _, _ in instances]
    systems = []
    for q, (m, (cfg, _, _, _)) in enumerate(zip(meshes, instances)):
        cap = 3 if q == 1 else 6000
        systems.append(api.System(m, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8,
                                  restart=500, max_iter=cap, max_refine=6))
    xs, st = api.solve_batch(systems, dirs, pols, raise_on_noconv=False)
    assert st[1].converged == 0
    for q, (x, s, (_, _, _, xr)) in enumerate(zip(xs, st, instances)):
        if q == 1:
            continue
        assert s.converged == 1
        assert _errs(x, xr).max() < 1e-5
    with pytest.raises(api.L.MtfError):
        api.solve_batch(systems, dirs, pols)
