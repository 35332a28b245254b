"""Oracle near field (Stratton-Chu representation, Eq. 8), pinned without
reference to its own formulas:

* in Omega_0 the near field times R exp(-i k0 R) tends to the far field
  (whose formula is pinned by the Mie series) with an O(1/R) error;
* block 0's representation at points inside the scatterer is -E_inc (the
  incident field's representation from the complement, with both traces
  changing sign with the normal), converging under mesh refinement;
* block i's representation at points outside Omega_i vanishes (the second
  case of Eq. 8), converging under mesh refinement."""
import numpy as np
import pytest

import mtf_inputs as mi
from oracle.mtf import MTFSystem
from oracle.nearfield import representation
from tests.oracle_helpers import skeleton_of

PIN = np.array([[0.1, 0.2, -0.1], [0.0, 0.0, 0.4], [-0.3, 0.1, 0.2]])   # inside the unit sphere
POUT = np.array([[0.0, 0.0, 2.0], [1.5, 0.5, 0.0], [0.0, -2.0, 1.0]])  # outside


@pytest.fixture(scope="module")
def spheres():
    out = {}
    for level in (1, 2):
        cfg = mi.config_sphere(level=level)
        sk = skeleton_of(cfg["mesh"])
        ref = MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"])
        x = ref.solve_lu(ref.rhs(cfg["dirs"], cfg["pols"]))[:, 0]
        out[level] = (cfg, ref, x)
    return out


def test_near_field_tends_to_the_far_field(spheres):
    cfg, ref, x = spheres[1]
    xh = np.array([[0.6, 0.0, 0.8], [0.0, 1.0, 0.0], [0.0, 0.0, -1.0]])
    finf = ref.farfield(x, xh)[:, :, 0]
    errs = []
    for R in (200.0, 800.0):
        e = representation(ref, x, R * xh, np.zeros(3, int))[:, :, 0] * R * np.exp(-1j * ref.k0 * R)
        errs.append(np.linalg.norm(e - finf) / np.linalg.norm(finf))
    assert errs[0] < 0.02
    assert 3.5 < errs[0] / errs[1] < 4.5, errs      # O(1/R)


def test_exterior_representation_inside_is_minus_incident_field(spheres):
    errs = []
    for level in (1, 2):
        cfg, ref, x = spheres[level]
        d, p = cfg["dirs"][0], cfg["pols"][0]
        einc = p[None, :] * np.exp(1j * ref.k0 * (PIN @ d))[:, None]
        e0 = representation(ref, x, PIN, np.zeros(len(PIN), int))[:, :, 0]
        errs.append(np.linalg.norm(e0 + einc) / np.linalg.norm(einc))
    assert errs[1] < 1e-4 and errs[1] < errs[0] / 4, errs


def test_interior_representation_vanishes_outside(spheres):
    ratios = []
    for level in (1, 2):
        cfg, ref, x = spheres[level]
        ein = representation(ref, x, PIN, np.ones(len(PIN), int))[:, :, 0]
        eout = representation(ref, x, POUT, np.ones(len(POUT), int))[:, :, 0]
        assert np.linalg.norm(ein) > 0.5 * len(PIN) ** 0.5
        ratios.append(np.linalg.norm(eout) / np.linalg.norm(ein))
    assert ratios[1] < 1e-4 and ratios[1] < ratios[0] / 4, ratios
