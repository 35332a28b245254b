"""GPU (FP64 path) vs oracle parity through the C-ABI.

Tolerance: relative 1e-10 for the FP64 path (norm-wise, ||gpu - ref|| /
||ref||), the bound stated for the exact path.  Small cases compare every
output element; the full-size split-sphere workload compares sampled full
matrix rows and sampled rows of M x that the oracle computes one by one."""
import numpy as np
import pytest
import torch

import mtf_inputs as mi
from oracle.mtf import MTFSystem
from oracle.operators import block_rows, transmission_gram
from tests.oracle_helpers import skeleton_of, sphere_system, rcs_plane

pytestmark = pytest.mark.gpu
TOL = 1e-10


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


def _case(cache, name):
    if ("gpucase", name) in cache:
        return cache[("gpucase", name)]
    if name == "sphere":
        cfg, sk, ref = sphere_system(cache, 2)
    elif name == "split":
        cfg = mi.config_split_sphere(rings=4, k0=2.0)
        sk = skeleton_of(cfg["mesh"])
        ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    elif name == "cubes":
        cfg = mi.config_cube2(n=2, k0=3.0, n_dirs=3)
        sk = skeleton_of(cfg["mesh"])
        ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    elif name == "uvodd":
        # odd block size (N = 567): odd piece lengths and padded rows in the
        # streaming kernels
        cfg = dict(mesh=mi.uv_sphere(10, 21), k0=1.5, eps_r=np.array([1.0, 2.5]), mu_r=np.array([1.0, 1.0]),
                   dirs=np.array([[0.0, 0.0, 1.0]]), pols=np.array([[1.0, 0.0, 0.0]], dtype=np.complex128))
        sk = skeleton_of(cfg["mesh"])
        ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    cache[("gpucase", name)] = (cfg, sk, ref)
    return cfg, sk, ref


@pytest.mark.parametrize("name", ["sphere", "split", "cubes"])
def test_blocks_match_oracle(api, oracle_cache, name):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    for i in range(sk.n_domains):
        T, K = (t.cpu().numpy() for t in sysg.block(i))
        assert rel(T, ref.T[i]) < TOL, (i, rel(T, ref.T[i]))
        assert rel(K, ref.K[i]) < TOL, (i, rel(K, ref.K[i]))


@pytest.mark.parametrize("name", ["sphere", "split", "cubes"])
@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_matvec_and_rhs_match_oracle(api, oracle_cache, name, nrhs):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    rng = np.random.default_rng(nrhs)
    x = rng.standard_normal((nrhs, sk.n_total)) + 1j * rng.standard_normal((nrhs, sk.n_total))
    y = sysg.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    yr = ref.matvec(x.T).T
    assert rel(y, yr) < TOL
    dirs, pols = mi.plane_wave_batch(max(1, nrhs // 2))
    dirs, pols = dirs[:nrhs], pols[:nrhs]
    if len(dirs) < nrhs:
        dirs, pols = np.repeat(dirs, nrhs, 0)[:nrhs], np.repeat(pols, nrhs, 0)[:nrhs]
    b = sysg.rhs(dirs, pols).cpu().numpy()
    assert rel(b, ref.rhs(dirs, pols).T) < TOL


@pytest.mark.parametrize("name", ["sphere", "split"])
def test_solve_and_farfield_match_oracle_lu(api, oracle_cache, name):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-12, restart=2000, max_iter=4000)
    x, st = sysg.solve(cfg["dirs"], cfg["pols"])
    xr = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))
    assert st.converged == 1 and st.rel_residual <= 1e-12
    assert rel(x.cpu().numpy().T, xr) < TOL
    obs = rcs_plane(37)
    f = sysg.farfield(x, obs).cpu().numpy()          # (nrhs, nobs, 3)
    fr = ref.farfield(xr, obs).transpose(2, 0, 1)
    assert rel(f, fr) < TOL


NEAR_POINTS = {
    "sphere": (np.array([[0.0, 0.0, 2.0], [1.5, 0.5, 0.0], [0.1, 0.2, -0.1], [0.0, 0.0, 0.4]]), [0, 0, 1, 1]),
    "split": (np.array([[0.0, 0.0, 2.0], [1.2, 0.9, 0.3], [0.1, 0.2, 0.4], [-0.3, 0.0, 0.5], [0.2, -0.1, -0.4],
                        [0.0, 0.3, -0.5]]), [0, 0, 1, 1, 2, 2]),
}


@pytest.mark.parametrize("name", ["sphere", "split"])
def test_nearfield_matches_oracle(api, oracle_cache, name):
    """U = H(gamma_D U) + E(gamma_N U) (Eq. 8) at points of every subdomain,
    from the same (oracle LU) solution on both sides."""
    from oracle.nearfield import representation
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    xr = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))
    pts, dom = NEAR_POINTS[name]
    f = sysg.nearfield(torch.from_numpy(np.ascontiguousarray(xr.T)).cuda(), pts, dom).cpu().numpy()
    fr = representation(ref, xr, pts, np.array(dom)).transpose(2, 0, 1)
    assert rel(f, fr) < TOL, rel(f, fr)


def test_degenerate_inputs_are_rejected(api, oracle_cache):
    from paper_2502_10907_gb300 import _lib as L
    cfg, sk, ref = _case(oracle_cache, "sphere")
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    x = torch.zeros((1, sk.n_total), dtype=torch.complex128, device="cuda")
    with pytest.raises(L.MtfError):
        L.mtf_matvec(sysg.handle, x, x, 1)            # aliasing
    y = torch.empty_like(x)
    with pytest.raises(L.MtfError):
        L.mtf_matvec(sysg.handle, x, y, 0)            # empty batch
    with pytest.raises(L.MtfError):
        sysg.rhs(np.array([[0.0, 0.0, 2.0]]), np.array([[1.0, 0, 0]], dtype=complex))  # not unit
    with pytest.raises(L.MtfError):
        api.System(mesh, -1.0, cfg["eps_r"], cfg["mu_r"])
    # zero incident field -> zero solution, converged at once
    xs, st = sysg.solve(np.array([[0.0, 0.0, 1.0]]), np.zeros((1, 3), dtype=complex))
    assert st.converged == 1 and float(xs.abs().max()) == 0.0


def test_full_size_split_sphere_sampled_rows(api):
    """Split sphere, 2178 skeleton triangles (the benchmark workload), in
    the benchmark's launch configuration: sampled full rows of T_i, K_i and
    sampled rows of M x against the oracle."""
    cfg = mi.config_split_sphere()
    sk = skeleton_of(cfg["mesh"])
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"], assemble=False)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, sk.n_total)) + 1j * rng.standard_normal((2, sk.n_total))
    y = sysg.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    for i in range(sk.n_domains):
        rows = np.sort(rng.choice(sk.N[i], 3, replace=False))
        rows[0] = 0
        Tr, Kr = block_rows(sk, i, ref.k[i], rows)
        T, K = (t.cpu().numpy()[rows] for t in sysg.block(i))
        assert rel(T, Tr) < TOL and rel(K, Kr) < TOL
        Di, Ni = sk.block_slices(i)
        r = ref.rho[i]
        yD = 2 * (Kr @ x[:, Di].T + (Tr @ x[:, Ni].T) / r)
        yN = 2 * (-r * (Tr @ x[:, Di].T) + Kr @ x[:, Ni].T)
        for j in sk.Lambda[i]:
            Gij = transmission_gram(sk, i, j)[rows]
            Dj, Nj = sk.block_slices(j)
            yD += Gij @ x[:, Dj].T
            yN += Gij @ x[:, Nj].T
        assert rel(y[:, Di][:, rows], yD.T) < TOL
        assert rel(y[:, Ni][:, rows], yN.T) < TOL


# ---------------------------------------------------------------------------
# mixed precision: FP32 regular pairs and storage, FP64 singular pairs,
# FP32-matvec FGMRES inside FP64 iterative refinement.  Stated bound: 1e-5
# relative error of solutions and far fields vs the FP64 oracle; the
# assembled blocks carry FP32 rounding (bound 2e-6 norm-wise).
# ---------------------------------------------------------------------------
MIXED_TOL = 1e-5


@pytest.mark.parametrize("name", ["sphere", "split", "cubes"])
def test_mixed_blocks_match_oracle(api, oracle_cache, name):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1)
    for i in range(sk.n_domains):
        T, K = (t.cpu().numpy() for t in sysg.block(i))
        assert rel(T, ref.T[i]) < 2e-6, (i, rel(T, ref.T[i]))
        assert rel(K, ref.K[i]) < 2e-6, (i, rel(K, ref.K[i]))


@pytest.mark.parametrize("name", ["sphere", "split", "cubes"])
def test_mixed_solve_and_farfield_within_1e5_of_oracle(api, oracle_cache, name):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, tol=1e-8, restart=2000,
                      max_iter=6000, max_refine=6)
    x, st = sysg.solve(cfg["dirs"], cfg["pols"])
    xr = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))
    assert st.converged == 1
    errs = np.linalg.norm(x.cpu().numpy().T - xr, axis=0) / np.linalg.norm(xr, axis=0)
    assert errs.max() < MIXED_TOL, errs
    obs = rcs_plane(37)
    f = sysg.farfield(x, obs).cpu().numpy()
    fr = ref.farfield(xr, obs).transpose(2, 0, 1)
    assert rel(f, fr) < MIXED_TOL


# ---------------------------------------------------------------------------
# block-OSRC preconditioner (Eq. 19).  The apply uses an FP32 eigensolver and
# FP32 passes: bound 1e-4 against the FP64 oracle operator.  Preconditioned
# solves converge to the same solution (1e-10 FP64, 1e-5 mixed).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["sphere", "split", "uvodd"])
def test_osrc_apply_matches_oracle(api, oracle_cache, name):
    from oracle.osrc import BlockOSRC
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precond=1)
    P = BlockOSRC(sk, ref.k, ref.rho)
    rng = np.random.default_rng(11)
    r = rng.standard_normal((3, sk.n_total)) + 1j * rng.standard_normal((3, sk.n_total))
    z = sysg.precond(torch.from_numpy(r).cuda()).cpu().numpy()
    zr = np.stack([P.apply(rr) for rr in r])
    assert rel(z, zr) < 1e-4


@pytest.mark.parametrize("name", ["sphere", "split"])
def test_osrc_preconditioned_solves(api, oracle_cache, name):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    xr = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))
    plain = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-6, restart=2000, max_iter=4000)
    _, st0 = plain.solve(cfg["dirs"], cfg["pols"])
    pre = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-6, restart=2000, max_iter=4000,
                     precond=1)
    _, st1 = pre.solve(cfg["dirs"], cfg["pols"])
    assert st1.iterations * 2 < st0.iterations, (st0.iterations, st1.iterations)
    exact = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-12, restart=2000, max_iter=4000,
                       precond=1)
    x, st = exact.solve(cfg["dirs"], cfg["pols"])
    assert rel(x.cpu().numpy().T, xr) < TOL
    mixed = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], tol=1e-8, restart=500, max_iter=4000,
                       precond=1, precision=1, max_refine=6)
    xm, stm = mixed.solve(cfg["dirs"], cfg["pols"])
    errs = np.linalg.norm(xm.cpu().numpy().T - xr, axis=0) / np.linalg.norm(xr, axis=0)
    assert stm.converged == 1 and errs.max() < MIXED_TOL, errs


# ---------------------------------------------------------------------------
# mixed precision with restarted inner cycles: the FP32-basis FGMRES cycles
# end on the restart length or the inner tolerance, and every cycle starts
# from an FP64 residual; 6 right-hand sides exercise the 4 + 2 column chunks
# of the FP32 matvec and OSRC passes.  Restart lengths are ones with which
# restarted GMRES on this system converges in the oracle's own GMRES (the
# unpreconditioned system needs ~1450 iterations of full GMRES, and restarts
# of 200 still stagnate in FP64 there, so that case runs one long cycle per
# refinement step).  Same 1e-5 bound against the oracle LU.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("block", [0, 1])
@pytest.mark.parametrize("precond,restart", [(0, 2000), (1, 50)])
def test_mixed_restarted_six_rhs(api, oracle_cache, precond, restart, block):
    cfg, sk, ref = _case(oracle_cache, "split")
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    dirs, pols = mi.plane_wave_batch(3)
    xr = ref.solve_lu(ref.rhs(dirs, pols))
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, tol=1e-8, restart=restart,
                      max_iter=8000, max_refine=8, precond=precond, block_krylov=block)
    x, st = sysg.solve(dirs, pols)
    assert st.converged == 1
    assert st.restarts >= 2, st.restarts
    errs = np.linalg.norm(x.cpu().numpy().T - xr, axis=0) / np.linalg.norm(xr, axis=0)
    assert errs.max() < MIXED_TOL, errs


# ---------------------------------------------------------------------------
# FP32 entry points of the mixed inner solver: the matvec on the tensor cores
# (FP16 hi + lo split, up to 32 right-hand sides per pass) and the FMA stream
# (rows cut into pieces of <= 512 columns, 4 right-hand sides per pass), and
# the FP32 OSRC apply.  Bound: 1e-5 norm-wise and entry by entry (relative to
# the largest entry) against the FP64 oracle for the matvec, 1e-4 for the
# OSRC apply as for its FP64-vector entry.  nrhs 1, 3, 6, 16 and 40 cover
# every column-chunk width of the FMA stream (1..4) and every input width of
# the tensor-core kernel (16, 32, 64, 128 columns, two passes for 40).
# ---------------------------------------------------------------------------
def _rand_c64(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def test_recycled_second_cycle_matches_oracle_with_fewer_iterations(api, oracle_cache):
    """The second inner cycle started from the first cycle's space (GCRO
    recycling) reaches the oracle's solution like a plain restart, in fewer
    iterations (the plain restart repeats GMRES's slow start)."""
    cfg, sk, ref = _case(oracle_cache, "split")
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    xr = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))
    its = {}
    for rec in (0, 1):
        sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8,
                          restart=400, max_iter=4000, max_refine=6, recycle=rec, block_krylov=0)
        x, st = sysg.solve(cfg["dirs"], cfg["pols"])
        assert st.converged == 1 and st.restarts >= 2
        errs = np.linalg.norm(x.cpu().numpy().T - xr, axis=0) / np.linalg.norm(xr, axis=0)
        assert errs.max() < MIXED_TOL, (rec, errs)
        its[rec] = st.iterations
    assert its[1] < 0.8 * its[0], its


@pytest.mark.parametrize("tensor", [1, 0])
@pytest.mark.parametrize("name", ["sphere", "split", "cubes", "uvodd"])
@pytest.mark.parametrize("nrhs", [1, 3, 6, 16, 36, 40])
def test_matvec_f32_matches_oracle(api, oracle_cache, name, nrhs, tensor):
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, mv_tensor=tensor)
    x = _rand_c64(np.random.default_rng(nrhs), (nrhs, sk.n_total))
    y = sysg.matvec_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    yr = np.stack([ref.matvec(xx.astype(np.complex128)) for xx in x])
    assert rel(y, yr) < 1e-5, rel(y, yr)
    # entry by entry: no entry is off by more than 1e-5 of the largest
    assert np.abs(y - yr).max() < 1e-5 * np.abs(yr).max(), np.abs(y - yr).max() / np.abs(yr).max()
    # repeated launches give identical results (schedule-independent sums)
    y2 = sysg.matvec_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y, y2)


def test_matvec_f32_full_size_sampled_rows(api):
    """Benchmark workload (rows of ~2200 columns in 5 pieces each), nrhs 2."""
    cfg = mi.config_split_sphere()
    sk = skeleton_of(cfg["mesh"])
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"], assemble=False)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1)
    rng = np.random.default_rng(8)
    x = _rand_c64(rng, (2, sk.n_total))
    y = sysg.matvec_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    xd = x.astype(np.complex128)
    for i in range(sk.n_domains):
        rows = np.sort(rng.choice(sk.N[i], 4, replace=False))
        Tr, Kr = block_rows(sk, i, ref.k[i], rows)
        Di, Ni = sk.block_slices(i)
        r = ref.rho[i]
        yD = 2 * (Kr @ xd[:, Di].T + (Tr @ xd[:, Ni].T) / r)
        yN = 2 * (-r * (Tr @ xd[:, Di].T) + Kr @ xd[:, Ni].T)
        for j in sk.Lambda[i]:
            Gij = transmission_gram(sk, i, j)[rows]
            Dj, Nj = sk.block_slices(j)
            yD += Gij @ xd[:, Dj].T
            yN += Gij @ xd[:, Nj].T
        assert rel(y[:, Di][:, rows], yD.T) < 1e-5
        assert rel(y[:, Ni][:, rows], yN.T) < 1e-5


@pytest.mark.parametrize("name", ["sphere", "split", "uvodd"])
@pytest.mark.parametrize("nrhs", [5, 36])
def test_osrc_apply_f32_matches_oracle(api, oracle_cache, name, nrhs):
    from oracle.osrc import BlockOSRC
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    P = BlockOSRC(sk, ref.k, ref.rho)
    r = _rand_c64(np.random.default_rng(12), (nrhs, sk.n_total))
    zr = np.stack([P.apply(rr.astype(np.complex128)) for rr in r])
    # FP32 T~: FP32 storage and sums; FP16 copy: entries rounded to 11
    # significant bits of the block's largest entry (2^-12 relative at most),
    # applied by the tensor cores (FP16 hi + lo inputs, up to 32 per pass) or
    # by the mma.sync stream (FP16 inputs, 4 per pass)
    for half, tensor, tol in ((0, 0, 1e-4), (1, 1, 1e-3), (1, 0, 1e-3)):
        sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precond=1, precision=1, osrc_half=half,
                          mv_tensor=tensor)
        z = sysg.precond_f32(torch.from_numpy(r).cuda()).cpu().numpy()
        assert rel(z, zr) < tol, (half, tensor, rel(z, zr))
        assert np.abs(z - zr).max() < tol * np.abs(zr).max(), (half, tensor)



# ---------------------------------------------------------------------------
# block-OSRC Type 2 (Sec. 5.4; reading: modal symbols with the phase of the
# EtM principal symbols, T~2 = i R with R real symmetric).  The wide
# tensor-core apply streams R alone in FP16 (real input chunks, 64 columns
# per chunk, odd N padded), the narrow applies the complex copy whose real
# part is zero; both against the oracle's Type-2 operator.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["split", "uvodd", "cubes"])
def test_osrc_type2_apply_matches_oracle(api, oracle_cache, name):
    from oracle.osrc import BlockOSRC
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    P2 = BlockOSRC(sk, ref.k, ref.rho, osrc_type=2)
    P1 = BlockOSRC(sk, ref.k, ref.rho)
    rng = np.random.default_rng(13)
    r = rng.standard_normal((3, sk.n_total)) + 1j * rng.standard_normal((3, sk.n_total))
    s64 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precond=1, osrc_type=2)
    z = s64.precond(torch.from_numpy(r).cuda()).cpu().numpy()
    zr = np.stack([P2.apply(rr) for rr in r])
    assert rel(z, zr) < 1e-4
    # Type 2 is a different operator from Type 1 (not a relabelling)
    assert rel(np.stack([P1.apply(rr) for rr in r]), zr) > 1e-2
    s32 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precond=1, precision=1, osrc_type=2)
    for nrhs in (3, 9, 36):
        r32 = _rand_c64(rng, (nrhs, sk.n_total))
        zr = np.stack([P2.apply(rr.astype(np.complex128)) for rr in r32])
        z = s32.precond_f32(torch.from_numpy(r32).cuda()).cpu().numpy()
        assert rel(z, zr) < 1e-3, (nrhs, rel(z, zr))
        assert np.abs(z - zr).max() < 1e-3 * np.abs(zr).max(), nrhs


@pytest.mark.parametrize("name", ["split", "cubes"])
def test_osrc_type2_solves_to_the_same_solution(api, oracle_cache, name):
    """Eight plane waves through the mixed block solver (the wide Type-2
    apply inside): both types reach the oracle's LU solution within 1e-5,
    and Type 2 needs at most 1.5x Type 1's iterations."""
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    dirs, pols = mi.plane_wave_batch(4)
    xr = ref.solve_lu(ref.rhs(dirs, pols))
    its = {}
    for t in (1, 2):
        sysg = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, precond=1, tol=1e-8, restart=500,
                          max_iter=4000, max_refine=6, osrc_type=t)
        x, st = sysg.solve(dirs, pols)
        errs = np.linalg.norm(x.cpu().numpy().T - xr, axis=0) / np.linalg.norm(xr, axis=0)
        assert st.converged == 1 and errs.max() < MIXED_TOL, (t, errs)
        its[t] = st.iterations
    assert its[2] <= 1.5 * its[1], its
    with pytest.raises(api.L.MtfError):
        api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precond=1, osrc_type=3)

def test_f32_entries_reject_wrong_systems(api, oracle_cache):
    cfg, sk, ref = _case(oracle_cache, "sphere")
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    sys64 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    x = torch.zeros((1, sk.n_total), dtype=torch.complex64, device="cuda")
    with pytest.raises(api.L.MtfError):
        sys64.matvec_f32(x)
    with pytest.raises(api.L.MtfError):
        sys64.precond_f32(x)


@pytest.mark.parametrize("name", ["split", "cubes"])
def test_mixed_residual_matvec_is_exact_for_the_stored_operator(api, oracle_cache, name):
    """The refinement residual of the mixed path applies the FP32-stored
    operator to an FP64 vector with double-float sums (a split input and
    error-free products and two-sums; option residual_df, default on) or with
    FP64 sums.  Against the same stored blocks applied in FP64 by numpy (the
    exchange part from the oracle), both must agree to near FP64 accuracy, far
    below the FP32 storage error.  Each system is compared with its own
    blocks: the FP32 assembly adds singular pairs atomically, so two
    assemblies may differ in the last bit."""
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    rng = np.random.default_rng(31)
    x = rng.standard_normal((3, sk.n_total)) + 1j * rng.standard_normal((3, sk.n_total))
    for df, tol in ((1, 1e-12), (0, 1e-13)):
        s32 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, residual_df=df)
        y = s32.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
        yr = ref.matvec(x.T).T                          # FP64 blocks + exchange
        for i in range(sk.n_domains):                   # swap in the stored FP32 blocks
            T, K = (t.cpu().numpy() for t in s32.block(i))
            dT, dK, r = T - ref.T[i], K - ref.K[i], ref.rho[i]
            Di, Ni = sk.block_slices(i)
            yr[:, Di] += (2.0 * (dK @ x[:, Di].T + (dT @ x[:, Ni].T) / r)).T
            yr[:, Ni] += (2.0 * (-r * (dT @ x[:, Di].T) + dK @ x[:, Ni].T)).T
        assert rel(y, yr) < tol, (df, rel(y, yr))
        assert rel(y, ref.matvec(x.T).T) > 1e-9      # the FP32 storage error is visible


@pytest.mark.parametrize("name", ["split", "cubes"])
def test_residual_fp64_matvec_matches_the_fp64_blocks(api, oracle_cache, name):
    """residual_fp64: the mixed system keeps the FP64 blocks as FP32 pairs and
    applies them with double-float sums (the refinement residual and
    mtf_matvec); against the FP64 system's FP64 matvec of the same blocks the
    difference is the double-float rounding, far below the FP32 entry error."""
    cfg, sk, ref = _case(oracle_cache, name)
    mesh = api.Mesh.from_inputs(cfg["mesh"])
    s64 = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    sdf = api.System(mesh, cfg["k0"], cfg["eps_r"], cfg["mu_r"], precision=1, residual_fp64=1)
    rng = np.random.default_rng(17)
    x = rng.standard_normal((5, sk.n_total)) + 1j * rng.standard_normal((5, sk.n_total))
    xt = torch.from_numpy(x).cuda()
    y64 = s64.matvec(xt).cpu().numpy()
    ydf = sdf.matvec(xt).cpu().numpy()
    assert rel(ydf, y64) < 1e-12, rel(ydf, y64)
    assert np.abs(ydf - y64).max() < 1e-12 * np.abs(y64).max()
