"""Pins of the oracle's block-OSRC preconditioner (Sec. 4.4, Eq. 19).

The OSRC operator only changes iteration counts, never the solution; its
pins are the Pade approximation of the square root (against the principal
square root away from the rotated branch cut), the structure of the RWG
div-div matrix, and the effect the paper reports: block-OSRC speeds up GMRES
by more than 3x (Sec. 5.3)."""
import numpy as np
import pytest

import mtf_inputs as mi
from oracle.osrc import (pade_sqrt, pade_coefficients, divdiv_matrix, BlockOSRC, gmres_iterations,
                         p1_matrices, loop_map)
from oracle.operators import mass_matrix
from tests.oracle_helpers import sphere_system, skeleton_of


def test_pade_sqrt_converges_to_principal_root():
    z = np.concatenate([np.linspace(-0.9, 4.0, 40), np.linspace(-0.9, 4.0, 40) + 0.3j])
    e4 = np.abs(pade_sqrt(z, 4) - np.sqrt(1 + z)).max()
    e8 = np.abs(pade_sqrt(z, 8) - np.sqrt(1 + z)).max()
    assert e4 < 3e-2 and e8 < 1e-3 and e8 < e4 / 20
    assert np.abs(pade_sqrt(z, 16) - np.sqrt(1 + z)).max() < 1e-6   # exponential in N_p
    C0, A, B = pade_coefficients(4, np.pi / 2)
    assert abs(C0 + A.sum() * 0 - pade_sqrt(0.0, 4)) < 1e-15     # P(0) = C0
    assert abs(C0 - 1.0) < 1e-3
    # evanescent side (rotated cut): finite, follows i sqrt(|z| - 1)
    z = -np.linspace(2.0, 6.0, 9) + 1e-3j
    assert np.abs(pade_sqrt(z, 8) - np.sqrt(1 + z)).max() < 5e-2


def test_divdiv_matrix_rank_and_symmetry():
    sk = skeleton_of(mi.icosphere(1))
    D = divdiv_matrix(sk, 0)
    G = mass_matrix(sk, 0)
    assert np.allclose(D, D.T) and np.allclose(G, G.T)
    ev = np.linalg.eigvalsh(D)
    T = len(sk.tris[0])
    # div maps RWG onto zero-mean piecewise constants: rank T - 1
    assert np.sum(ev > 1e-10 * ev.max()) == T - 1
    assert np.all(np.linalg.eigvalsh(G) > 0)


def test_loop_map_is_divergence_free_and_isometric():
    """L maps nodal P1 values to the RWG coefficients of n x grad(phi):
    div L phi = 0 exactly (D L = 0) and ||L phi||_G^2 = phi^T S phi."""
    sk = skeleton_of(mi.split_sphere(3))
    for i in range(sk.n_domains):
        verts, pos, S, M = p1_matrices(sk, i)
        L = loop_map(sk, i, pos)
        D = divdiv_matrix(sk, i)
        G = mass_matrix(sk, i)
        assert np.abs(D @ L).max() < 1e-12 * np.abs(D).max()
        assert np.abs(L.T @ G @ L - S).max() < 1e-12 * np.abs(S).max()
        # P1 Laplace-Beltrami: constants in the kernel, M symmetric positive definite
        assert np.abs(S @ np.ones(len(verts))).max() < 1e-12
        assert np.all(np.linalg.eigvalsh(M) > 0)


def test_block_osrc_speeds_up_gmres(oracle_cache):
    cfg, sk, ref = sphere_system(oracle_cache, 2)
    M = ref.matrix()
    b = ref.rhs(cfg["dirs"], cfg["pols"])[:, 0]
    xs = np.linalg.solve(M, b)
    P = BlockOSRC(sk, ref.k, ref.rho)
    x0, it0, c0 = gmres_iterations(M, b, 1e-5, 100, 1500)
    x1, it1, c1 = gmres_iterations(M, b, 1e-5, 100, 1500, P=P.matrix())
    assert c1 and it1 * 3 < it0, (it0, it1)
    # the preconditioner changes the iterations, not the solution
    assert np.linalg.norm(x1 - xs) / np.linalg.norm(xs) < 1e-3
    r = np.random.default_rng(0).standard_normal(sk.n_total) + 0j
    assert np.allclose(P.apply(r), P.matrix() @ r)


def test_block_osrc_on_genus_one_boundaries():
    """Concentric cuboids (M = 2): the outer ring's boundary is a torus
    (genus 1), so its RWG space holds 2 discrete harmonic fields beside the
    irrotational and loop modes (Euler: N - (T - 1) - (V - 1) = 2 g).  The
    completed basis is G-orthonormal, the harmonic fields are divergence-free,
    T~ stays symmetric, and block-OSRC makes GMRES converge where the plain
    iteration stalls (the behaviour the paper reports for the cuboids)."""
    cfg = mi.config_concentric_cuboids(2, h=0.6)
    sk = skeleton_of(cfg["mesh"])
    from oracle.mtf import MTFSystem
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
    P = BlockOSRC(sk, ref.k, ref.rho)
    assert P.nh == [0, 0, 2]
    for i in range(sk.n_domains):
        G, D, W = mass_matrix(sk, i), divdiv_matrix(sk, i), P.W[i]
        assert W.shape == (sk.N[i], sk.N[i])
        assert np.abs(W.T @ G @ W - np.eye(sk.N[i])).max() < 1e-10
        if P.nh[i]:
            H = W[:, -P.nh[i]:]
            assert np.abs(H.T @ D @ H).max() < 1e-12 * np.abs(D).max()
        assert np.abs(P.Ttil[i] - P.Ttil[i].T).max() < 1e-12 * np.abs(P.Ttil[i]).max()
    M = ref.matrix()
    b = ref.rhs(cfg["dirs"], cfg["pols"])[:, 0]
    _, it0, c0 = gmres_iterations(M, b, 1e-5, 100, 600)
    _, it1, c1 = gmres_iterations(M, b, 1e-5, 100, 600, P=P.matrix())
    assert c1 and not c0 and it1 < 300, (it0, it1)


def test_block_osrc_type2_modal_structure(oracle_cache):
    """Type 2 (Sec. 5.4; reading: the Type-1 symbols with their modulus kept
    and their phase set to that of the EtM principal symbols).  Pinned without
    the mode basis the oracle builds it from: T~2 is purely imaginary and
    symmetric; the eigenvalues of T~2 G (G the RWG Gram matrix) are the
    Type-2 symbols, so they have the moduli of the eigenvalues of T~1 G and
    are purely imaginary; exactly T_i - 1 of them (the rank of div on RWG_i)
    lie on the negative imaginary axis; and the eigenvectors on the positive
    axis are divergence-free (D v = 0: loops and harmonic fields), those on
    the negative axis are not."""
    cfg, sk, ref = sphere_system(oracle_cache, 2)
    P1 = BlockOSRC(sk, ref.k, ref.rho, Np=16)
    P2 = BlockOSRC(sk, ref.k, ref.rho, Np=16, osrc_type=2)
    for i in range(sk.n_domains):
        G, D = mass_matrix(sk, i), divdiv_matrix(sk, i)
        T1, T2 = P1.Ttil[i], P2.Ttil[i]
        assert np.abs(T2.real).max() == 0.0
        assert np.abs(T2 - T2.T).max() < 1e-12 * np.abs(T2).max()
        l1 = np.linalg.eigvals(T1 @ G)
        l2, V2 = np.linalg.eig(T2 @ G)
        assert np.abs(np.sort(np.abs(l2)) - np.sort(np.abs(l1))).max() < 1e-9 * np.abs(l1).max()
        assert np.abs(l2.real).max() < 1e-9 * np.abs(l2).max()
        neg = l2.imag < 0
        assert int(neg.sum()) == len(sk.tris[i]) - 1
        Dv = np.linalg.norm(D @ V2, axis=0) / (np.linalg.norm(D) * np.linalg.norm(V2, axis=0))
        assert Dv[~neg].max() < 1e-8 and Dv[neg].min() > 1e-6, (Dv[~neg].max(), Dv[neg].min())


def test_block_osrc_type2_keeps_the_solution_and_the_iterations(oracle_cache):
    """Type 2 changes the preconditioner, not the solution, and keeps the
    iteration count near Type 1's (the paper reports similar convergence):
    within 1.25x of Type 1 and more than 3x below plain GMRES on the sphere."""
    cfg, sk, ref = sphere_system(oracle_cache, 2)
    M = ref.matrix()
    b = ref.rhs(cfg["dirs"], cfg["pols"])[:, 0]
    xs = np.linalg.solve(M, b)
    its = []
    for t in (1, 2):
        P = BlockOSRC(sk, ref.k, ref.rho, Np=16, osrc_type=t)
        x, it, c = gmres_iterations(M, b, 1e-5, 100, 1500, P=P.matrix())
        assert c and np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-3
        its.append(it)
    _, it0, _ = gmres_iterations(M, b, 1e-5, 100, 1500)
    assert its[1] <= 1.25 * its[0] and 3 * its[1] < it0, (its, it0)
    with pytest.raises(ValueError):
        BlockOSRC(sk, ref.k, ref.rho, osrc_type=3)


def test_block_osrc_type2_on_genus_one_boundaries():
    """Type 2 on the concentric cuboids (M = 2; the outer ring is bounded by a
    torus with 2 discrete harmonic fields): T~2 stays purely imaginary and
    symmetric, T~2 G has exactly T_i - 1 eigenvalues on the negative
    imaginary axis (the irrotational modes) and the rest, the harmonic
    fields among them, on the positive axis, with the moduli of Type 1's."""
    cfg = mi.config_concentric_cuboids(2, h=0.6)
    sk = skeleton_of(cfg["mesh"])
    from oracle.mtf import MTFSystem
    ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"], assemble=False)
    P1 = BlockOSRC(sk, ref.k, ref.rho)
    P2 = BlockOSRC(sk, ref.k, ref.rho, osrc_type=2)
    assert P2.nh == [0, 0, 2]
    for i in range(sk.n_domains):
        G = mass_matrix(sk, i)
        T2 = P2.Ttil[i]
        assert np.abs(T2.real).max() == 0.0
        assert np.abs(T2 - T2.T).max() < 1e-12 * np.abs(T2).max()
        l1 = np.linalg.eigvals(P1.Ttil[i] @ G)
        l2 = np.linalg.eigvals(T2 @ G)
        assert np.abs(np.sort(np.abs(l2)) - np.sort(np.abs(l1))).max() < 1e-9 * np.abs(l1).max()
        assert int((l2.imag < 0).sum()) == len(sk.tris[i]) - 1
        assert int((l2.imag > 0).sum()) == sk.N[i] - (len(sk.tris[i]) - 1)
