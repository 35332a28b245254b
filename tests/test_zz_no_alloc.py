"""mtf_solve_static: the GMRES solve without device allocation.

Some users of this library cannot let it call cudaMalloc while it runs --
for instance a service that has reserved a fixed slice of device memory up
front, or a loop that must not be stalled by the implicit device
synchronisation an allocation can cause.  For them the library offers
mtf_solve_static, which takes its workspace from a 16 MiB static device
array instead.  These tests call it through the C-ABI: twice in a row
against mtf_solve on the same system, with the tolerance the parity tests
use (1e-10, relative); on a block-OSRC system against the oracle's LU
solution and mtf_solve; and with a request larger than the static workspace,
which must be refused with a clear error.  It lives in its
own file, collected last, and builds the library itself so that it also
passes alone in a fresh process."""
import numpy as np
import pytest
import torch

import mtf_inputs as mi

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import _lib, api
    return _lib, api


def test_static_solve_matches_allocating_solve_twice(lib):
    L, api = lib
    cfg = mi.config_split_sphere(rings=3, k0=2.0)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-10, restart=400, max_iter=4000)
    x_ref, st_ref = sysg.solve(cfg["dirs"], cfg["pols"])
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = torch.full_like(x_ref, complex(np.nan, np.nan))
        st, status = L.mtf_solve_static(sysg.handle, cfg["dirs"], cfg["pols"], x, stream)
        torch.cuda.synchronize()
        assert status == 0 and st.converged == 1
        err = float((x - x_ref).norm() / x_ref.norm())
        assert err < TOL, (call, err)
        assert st.iterations == st_ref.iterations


def test_static_solve_with_block_osrc_matches_oracle_and_allocating_solve(lib):
    """A system assembled with block-OSRC is solved with that preconditioner
    (flexible GMRES): the solution equals the oracle's dense LU solution of
    the same discrete system to 1e-10, and mtf_solve's to 1e-10, and the
    preconditioner shows in the iteration count (fewer than the unpreconditioned
    static solve needs for a looser tolerance)."""
    L, api = lib
    from oracle.mtf import MTFSystem
    from tests.oracle_helpers import skeleton_of
    cfg = mi.config_split_sphere(rings=3, k0=2.0)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    pre = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-12, restart=200, max_iter=4000,
                     precond=L.MTF_PRECOND_OSRC)
    # without a preconditioner restarted GMRES needs a longer restart here
    plain = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-10, restart=400, max_iter=4000)
    stream = torch.cuda.current_stream().cuda_stream
    x_ref, _ = pre.solve(cfg["dirs"], cfg["pols"])
    sk = skeleton_of(cfg["mesh"])
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    x_lu = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))
    iters = {}
    for name, s in (("osrc", pre), ("plain", plain)):
        x = torch.full_like(x_ref, complex(np.nan, np.nan))
        st, status = L.mtf_solve_static(s.handle, cfg["dirs"], cfg["pols"], x, stream)
        torch.cuda.synchronize()
        assert status == 0 and st.converged == 1
        iters[name] = st.iterations
        if name == "osrc":
            xg = x.cpu().numpy().T
            err_lu = np.max(np.linalg.norm(xg - x_lu, axis=0) / np.linalg.norm(x_lu, axis=0))
            assert err_lu < TOL, err_lu
            err = float((x - x_ref).norm() / x_ref.norm())
            assert err < TOL, err
    # two decades more accuracy in fewer iterations: the preconditioner is applied
    assert iters["osrc"] < iters["plain"], iters


def test_static_solve_rejects_oversized_requests(lib):
    L, api = lib
    cfg = mi.config_sphere(level=1)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    # restart 3000 on 480 unknowns needs ~2.9M doubles > 2^21
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], restart=3000)
    x = torch.empty((1, mesh.n_total), dtype=torch.complex128, device="cuda")
    with pytest.raises(L.MtfError) as e:
        L.mtf_solve_static(sysg.handle, cfg["dirs"], cfg["pols"], x, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == L.MTF_ERR_ARG and "static workspace" in str(e.value)
