"""Pins of the oracle's full MTF solve against physics: Mie series (P1),
O(h^2) convergence (Sec. 5.2), MTF(2) with a triple junction, reciprocity
(P4), energy balance (P5), jump errors (Table 1 metric)."""
import numpy as np
import pytest
import scipy.special as sps

import mtf_inputs as mi
from oracle.mie import mie_farfield, mie_coefficients, _riccati_bessel, _riccati_hankel
from oracle.mtf import MTFSystem
from oracle.quadrature import gauss_legendre
from tests.oracle_helpers import skeleton_of, sphere_system, rcs_plane, jump_l2


def _sphere_dirs(nt=16, nph=32):
    mu, wmu = gauss_legendre(nt)
    mu, wmu = 2 * mu - 1, 2 * wmu
    ph = 2 * np.pi * np.arange(nph) / nph
    M, P = np.meshgrid(mu, ph, indexing="ij")
    st = np.sqrt(1 - M ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), M], axis=-1).reshape(-1, 3)
    w = (wmu[:, None] * np.full(nph, 2 * np.pi / nph)[None, :]).ravel()
    return dirs, w


def test_riccati_bessel_against_library():
    for z in (0.3, 1.0, 2.83, 7.5):
        psi, dpsi = _riccati_bessel(12, z)
        n = np.arange(13)
        assert np.allclose(psi, z * sps.spherical_jn(n, z), rtol=1e-12, atol=1e-300)
        xi, dxi = _riccati_hankel(12, z)
        assert np.allclose(xi.imag, z * sps.spherical_yn(n, z), rtol=1e-12)


def test_mie_rayleigh_limit():
    """Small sphere: far field of the quasi-static dipole
    p = 4 pi a^3 (eps-1)/(eps+2) E0, E_inf = k^2/(4 pi) (xhat x p) x xhat."""
    k, a, eps = 1e-2, 1.0, 2.5
    d, p = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    obs = np.array([[0.6, 0.0, 0.8], [0.0, 1.0, 0.0], [-0.48, 0.6, 0.64], [1.0, 0.0, 0.0]])
    F = mie_farfield(k, a, eps, d, p, obs)
    alpha = 4 * np.pi * a ** 3 * (eps - 1) / (eps + 2)
    Fd = k ** 2 / (4 * np.pi) * alpha * np.cross(np.cross(obs, p), obs)
    assert np.abs(F - Fd).max() < 1e-3 * np.abs(Fd).max()


def test_mie_optical_theorem():
    """Lossless sphere: scattered power = extinction (forward amplitude)."""
    k, a, eps = 1.3, 1.0, 3.0
    d, p = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    dirs, w = _sphere_dirs(24, 48)
    F = mie_farfield(k, a, eps, d, p, dirs)
    sca = np.sum(w * np.sum(np.abs(F) ** 2, axis=1))
    ext = 4 * np.pi / k * np.imag(p @ mie_farfield(k, a, eps, d, p, d[None])[0])
    assert abs(sca - ext) < 1e-9 * ext


def _bem_vs_mie(cfg, sysm, x):
    obs = rcs_plane()
    F = sysm.farfield(x, obs)[:, :, 0]
    Fm = mie_farfield(cfg["k0"], 1.0, cfg["eps_r"][1], cfg["dirs"][0], cfg["pols"][0], obs)
    return np.linalg.norm(F - Fm) / np.linalg.norm(Fm)


def test_mtf1_sphere_matches_mie_with_h2_convergence(oracle_cache):
    errs = []
    for lvl in (1, 2):
        cfg, sk, sysm = sphere_system(oracle_cache, lvl)
        x = sysm.solve_lu(sysm.rhs(cfg["dirs"], cfg["pols"]))
        oracle_cache[("sphere_x", lvl)] = x
        errs.append(_bem_vs_mie(cfg, sysm, x))
    assert errs[0] < 0.13 and errs[1] < 0.035, errs
    assert errs[0] / errs[1] > 3.0, errs          # O(h^2): h halves -> error / 4


def test_matvec_equals_dense_matrix(oracle_cache):
    cfg, sk, sysm = sphere_system(oracle_cache, 1)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((sk.n_total, 2)) + 1j * rng.standard_normal((sk.n_total, 2))
    assert np.allclose(sysm.matvec(x), sysm.matrix() @ x, rtol=1e-13, atol=1e-13)


def _split_system(cache, rings, eps2=2.0):
    key = ("split", rings, eps2)
    if key not in cache:
        mesh = mi.split_sphere(rings)
        sk = skeleton_of(mesh)
        sysm = MTFSystem(sk, 1.0, [1.0, 2.0, eps2], [1.0, 1.0, 1.0])
        d, p = np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]], dtype=complex)
        x = sysm.solve_lu(sysm.rhs(d, p))
        cache[key] = (sk, sysm, x, d, p)
    return cache[key]


def test_mtf2_triple_junction_matches_mie_and_jumps_converge(oracle_cache):
    """MTF(2): the sphere split in two halves with the same material (the
    paper's Sec. 5.2 experiment) must reproduce the Mie far field, and the
    Dirichlet/Neumann jumps across Gamma_12 must shrink under refinement."""
    res = []
    for rings in (3, 5):
        sk, sysm, x, d, p = _split_system(oracle_cache, rings)
        obs = rcs_plane()
        F = sysm.farfield(x, obs)[:, :, 0]
        Fm = mie_farfield(1.0, 1.0, 2.0, d[0], p[0], obs)
        res.append((np.linalg.norm(F - Fm) / np.linalg.norm(Fm),) + tuple(jump_l2(sk, x, 1, 2)))
    (e3, jd3, jn3), (e5, jd5, jn5) = res
    assert e3 < 0.15 and e5 < 0.06, res
    assert e5 < 0.5 * e3 and jd5 < 0.7 * jd3 and jn5 < 0.7 * jn3, res
    assert max(jd5, jn5) < 0.1, res


def test_reciprocity_and_energy_balance(oracle_cache):
    """P4: q . F(xhat; d, p) = p . F(-d; -xhat, q); P5: lossless scatterer,
    scattered power equals extinction (optical theorem)."""
    sk, sysm, _, _, _ = _split_system(oracle_cache, 3, eps2=4.0)
    d1, p1 = np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0])
    x1 = np.array([0.48, -0.6, 0.64])
    q1 = np.cross(x1, np.array([0.0, 0.0, 1.0]))
    q1 /= np.linalg.norm(q1)
    dirs = np.stack([d1, -x1])
    pols = np.stack([p1, q1]).astype(complex)
    x = sysm.solve_lu(sysm.rhs(dirs, pols))
    Fa = sysm.farfield(x[:, :1], x1[None])[0, :, 0]
    Fb = sysm.farfield(x[:, 1:], -d1[None])[0, :, 0]
    lhs, rhs = q1 @ Fa, p1 @ Fb
    assert abs(lhs - rhs) < 0.02 * abs(lhs)
    sd, w = _sphere_dirs(16, 32)
    F = sysm.farfield(x[:, :1], sd)[:, :, 0]
    sca = np.sum(w * np.sum(np.abs(F) ** 2, axis=1))
    ext = 4 * np.pi / sysm.k0 * np.imag(p1 @ sysm.farfield(x[:, :1], d1[None])[0, :, 0])
    assert abs(sca - ext) < 0.05 * ext


def test_artificial_interfaces_leave_the_far_field():
    """Concentric cuboids of one material (Sec. 5.4: the domain-decomposition
    test of the paper): splitting the scatterer into 2 square rings adds
    interfaces between equal media, so MTF(2) must reproduce the far field of
    the undivided scatterer MTF(1) meshed on the same grid, to discretisation
    accuracy (the rings' boundaries are tori, their walls meet the top and
    bottom faces in junction lines)."""
    import mtf_inputs.meshes as mm
    h = 0.45
    cfg = mi.config_concentric_cuboids(2, h=h)
    r = mi.cuboid_radii(2)
    xs = mm._graded(sorted({-v for v in r[1:]} | {v for v in r[1:]}), h)
    zs = mm._graded([0.0, 1.0], h)
    one = mm.grid_partition(xs, xs, zs, np.ones((len(xs) - 1, len(xs) - 1, len(zs) - 1), dtype=int))
    far = []
    for mesh, eps in ((cfg["mesh"], cfg["eps_r"]), (one, np.array([1.0, 2.0]))):
        sk = skeleton_of(mesh)
        sysm = MTFSystem(sk, cfg["k0"], eps, np.ones(len(eps)))
        x = sysm.solve_lu(sysm.rhs(cfg["dirs"], cfg["pols"]))
        far.append(sysm.farfield(x, rcs_plane(91))[:, :, 0])
    d = np.linalg.norm(far[0] - far[1]) / np.linalg.norm(far[1])
    assert d < 0.02, d


def test_mtf1_agrees_with_pmchwt(oracle_cache):
    """MTF(1) and PMCHWT (Sec. 3.1, the PMCHWT remark): summing the two block
    rows of Problem 2 with u_1 = -u_0 gives (A_0 - A_1) u_0 = u_inc.  The RWG
    functions of block 1 are the negatives of block 0's on the shared surface,
    so in coefficients u_1 = +u_0 and the system reads (2 A_0 + 2 A_1) u = b_0.
    Solving it from the same blocks gives a far field that agrees with
    MTF(1)'s far below both formulations' distance to the Mie series, and the
    gap closes under refinement; the opposite sign gives a wrong field."""
    gaps = []
    for lvl in (1, 2):
        cfg, sk, ref = sphere_system(oracle_cache, lvl)
        b = ref.rhs(cfg["dirs"], cfg["pols"])[:, 0]
        x = ref.solve_lu(b[:, None])[:, 0]
        D0, N0 = sk.block_slices(0)

        def A2(i):
            T, K, r = ref.T[i], ref.K[i], ref.rho[i]
            return 2.0 * np.block([[K, T / r], [-r * T, K]])

        obs = rcs_plane()
        F = ref.farfield(x[:, None], obs)[:, :, 0]
        Fm = mie_farfield(cfg["k0"], 1.0, cfg["eps_r"][1], cfg["dirs"][0], cfg["pols"][0], obs)
        for sign in (1.0, -1.0):
            u = np.linalg.solve(A2(0) + sign * A2(1), np.concatenate([b[D0], b[N0]]))
            xp = np.zeros_like(x)
            xp[D0], xp[N0] = u[: len(u) // 2], u[len(u) // 2:]
            Fp = ref.farfield(xp[:, None], obs)[:, :, 0]
            gap = np.linalg.norm(Fp - F) / np.linalg.norm(F)
            if sign > 0:
                gaps.append(gap)
                mie = np.linalg.norm(F - Fm) / np.linalg.norm(Fm)
                assert gap < 1e-3 * mie, (lvl, gap, mie)
            else:
                assert gap > 0.5, (lvl, gap)
    assert gaps[1] < gaps[0] / 4, gaps
