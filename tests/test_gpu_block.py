"""Block flexible GMRES of the mixed-precision inner solver (one Krylov space
shared by all right-hand sides), through the C-ABI, against the oracle's LU
solution of the same discrete system, at the mixed path's bound (1e-5 per
right-hand side).

* The 4 x 4 x 4 cube partition at its coarsest grid (65 blocks) with 16
  plane waves: the block solve and the per-rhs solve both reach the LU
  solution, and the block solve needs fewer block steps than the per-rhs
  solve needs iterations (each block step applies the operator to all 16
  vectors at once, so this is also fewer operator applies in total).
* A batch with a repeated plane wave and a zero-amplitude one: the start
  block is rank deficient, the dependent and the zero column are deflated
  (their directions dropped), and every column still reaches its own LU
  solution; the zero column stays exactly zero."""
import numpy as np
import pytest
import torch

import mtf_inputs as mi
from oracle.mtf import MTFSystem
from tests.oracle_helpers import skeleton_of

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def cube4():
    cfg = mi.config_cube4(n=1, n_dirs=8)
    sk = skeleton_of(cfg["mesh"])
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    return cfg, sk, ref


def _errs(x, xr):
    x = x.cpu().numpy().T
    return np.linalg.norm(x - xr, axis=0) / np.linalg.norm(xr, axis=0)


def test_block_solve_16_rhs_matches_oracle_lu(api, cube4):
    cfg, sk, ref = cube4
    dirs, pols = cfg["dirs"], cfg["pols"]
    assert len(dirs) == 16
    xr = ref.solve_lu(ref.rhs(dirs, pols))
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    its = {}
    for block in (1, 0):
        s = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8, restart=500,
                       max_iter=6000, max_refine=6, block_krylov=block)
        x, st = s.solve(dirs, pols)
        assert st.converged == 1
        errs = _errs(x, xr)
        assert errs.max() < MIXED_TOL, (block, errs)
        its[block] = st.iterations
    assert its[1] < its[0], its


def test_block_solve_deflates_dependent_and_zero_columns(api, cube4):
    cfg, sk, ref = cube4
    d = cfg["dirs"][[0, 0, 3, 5]]
    p = np.array(cfg["pols"][[0, 0, 3, 5]], dtype=np.complex128)
    p[3] = 0.0                                          # zero amplitude
    xr = ref.solve_lu(ref.rhs(d, p))
    live = np.linalg.norm(xr, axis=0) > 0
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    s = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8, restart=500,
                   max_iter=6000, max_refine=6, block_krylov=1)
    x, st = s.solve(d, p)
    assert st.converged == 1
    lv = torch.from_numpy(live).to(x.device)
    errs = _errs(x[lv], xr[:, live])
    assert errs.max() < MIXED_TOL, errs
    assert torch.all(x[~lv] == 0)
    # the repeated wave gets the same solution as its twin
    assert float((x[0] - x[1]).abs().max()) <= 1e-5 * float(x[0].abs().max())


@pytest.mark.parametrize("nw", [20, 40])
def test_wide_block_solve_matches_oracle_lu(api, cube4, nw):
    """Blocks wider than 16 vectors: the wide triangular solves (solved
    entries in shared memory), Gram-Schmidt passes of up to 2 x 40 columns in
    groups of 64, tensor-core applies in passes of up to 32 waves."""
    cfg, sk, ref = cube4
    dirs = mi.fibonacci_directions(nw // 2)
    p1, p2 = mi.orthonormal_polarizations(dirs)
    dirs = np.concatenate([dirs, dirs])
    pols = np.concatenate([p1, p2]).astype(np.complex128)
    xr = ref.solve_lu(ref.rhs(dirs, pols))
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    s = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8, restart=300,
                   max_iter=6000, max_refine=6, block_krylov=1)
    x, st = s.solve(dirs, pols)
    assert st.converged == 1
    errs = _errs(x, xr)
    assert errs.max() < MIXED_TOL, errs
