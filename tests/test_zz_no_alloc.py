"""mtf_solve_static: the GMRES solve without device allocation.

Some users of this library cannot let it call cudaMalloc while it runs --
for instance a service that has reserved a fixed slice of device memory up
front, or a loop that must not be stalled by the implicit device
synchronisation an allocation can cause.  For them the library offers
mtf_solve_static, which takes its workspace from a 16 MiB static device
array instead.  This test calls it through the C-ABI twice in a row and
checks both results against mtf_solve on the same system, with the tolerance
the parity tests use (1e-10, relative), and checks that a request larger
than the static workspace is refused with a clear error.  It lives in its
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
