"""Pins of the skeleton processing (Algorithm 1) and the RWG tables."""
import json
import os

import numpy as np
import pytest

import mtf_inputs as mi
from oracle.skeleton import Skeleton
from tests.oracle_helpers import skeleton_of

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table2_signed_lists.json")


def _table2_meshes():
    grid_labels = np.zeros((2, 2, 1), dtype=np.int64)
    grid_labels[0, 1, 0], grid_labels[0, 0, 0], grid_labels[1, 0, 0], grid_labels[1, 1, 0] = 1, 2, 3, 4
    return {
        "dielectric": mi.two_disjoint_cubes(n=2),
        "triple_point": mi.cube_partition((2, 1, 1), n=2, size=(2.0, 1.0, 1.0)),
        "grid": mi.cube_partition((2, 2, 1), n=2, size=(2.0, 2.0, 1.0), cell_labels=grid_labels),
    }


@pytest.mark.parametrize("case", ["dielectric", "triple_point", "grid"])
def test_algorithm1_reproduces_table2(case):
    gold = json.load(open(GOLD))[case]
    sk = skeleton_of(_table2_meshes()[case])
    for i, lst in gold.items():
        assert sk.signed_interface_list(int(i)) == lst


def _edge_uses(F):
    uses = {}
    for t, (a, b, c) in enumerate(F):
        for (u, v) in ((a, b), (b, c), (c, a)):
            uses.setdefault((min(u, v), max(u, v)), []).append((u, v))
    return uses


@pytest.mark.parametrize("mesh", [mi.icosphere(1), mi.split_sphere(3), mi.cube_partition((2, 2, 1), 2),
                                  mi.cut_sphere([0.4, -0.3], 0.4)], ids=lambda m: m.name)
def test_swapped_subdomain_surfaces_are_closed_and_outward(mesh):
    sk = skeleton_of(mesh)
    T = sum(len(t) for t in sk.tris)
    assert T == 2 * len(sk.F)                      # every triangle is on two boundaries
    assert sum(sk.N) * 2 == 3 * T                  # closed surfaces: 3 T_i = 2 N_i
    for i in range(sk.n_domains):
        F = sk.F[sk.tris[i]].copy()
        F[sk.swap[i] < 0] = F[sk.swap[i] < 0][:, [0, 2, 1]]
        for e, uses in _edge_uses(F).items():
            assert len(uses) == 2 and uses[0] == uses[1][::-1], (i, e)   # consistent orientation
        # outward: the flux of x through Gamma_i is 3 vol > 0 for bounded domains
        n = sk.outward_normal(i)
        c = sk.V[sk.F[sk.tris[i]]].mean(axis=1)
        flux = np.sum(np.einsum("tn,tn->t", c, n) * sk.area[sk.tris[i]])
        assert (flux > 0) if i > 0 else (flux < 0)


def test_rwg_div_conforming_and_swap_antisymmetric():
    sk = skeleton_of(mi.split_sphere(3))
    for i in range(sk.n_domains):
        dof, sgn = sk.dof[i], sk.sign[i]
        for d in range(sk.N[i]):
            s = sgn[dof == d]
            assert len(s) == 2 and s.sum() == 0
        # normal component of the RWG function on its edge is +1 / -1 (flux s * l)
        loc = np.arange(len(sk.tris[i]))
        c = sk.rwg_coeff(i)
        v = sk.V[sk.F[sk.tris[i]]]
        for a in range(3):
            p, q = v[:, (a + 1) % 3], v[:, (a + 2) % 3]
            mid = 0.5 * (p + q)
            e = q - p
            tnorm = sk.normal[sk.tris[i]]
            conormal = np.cross(e, tnorm)
            conormal /= np.linalg.norm(conormal, axis=1, keepdims=True)
            conormal *= np.sign(np.einsum("tn,tn->t", conormal, mid - v[:, a]))[:, None]
            flux = c[:, a] * np.einsum("tn,tn->t", mid - v[:, a], conormal)
            assert np.allclose(flux, sgn[:, a])
    # on a triangle of Gamma_ij the RWG_i and RWG_j functions of an edge are opposite
    pos = {i: {t: p for p, t in enumerate(sk.tris[i])} for i in range(sk.n_domains)}
    for t in range(len(sk.F)):
        i, j = sk.L[t]
        assert np.all(sk.sign[i][pos[i][t]] == -sk.sign[j][pos[j][t]])
