"""CPU tests of the C-ABI library: it loads, exports every entry point that
include/mtf.h declares, and its host-side skeleton processing (Algorithm 1,
RWG tables, pair classification) agrees with the oracle.  No compute call
is made without a GPU."""
import os
import re

import numpy as np
import pytest

import mtf_inputs as mi
from tests.oracle_helpers import skeleton_of
from oracle.operators import classify_pairs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_10907_gb300.build import build
    build()
    import paper_2502_10907_gb300 as P
    return P


def _declared():
    src = open(os.path.join(ROOT, "include", "mtf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mtf_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    import ctypes
    so = ctypes.CDLL(lib._lib.lib_path())
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib._lib.exported_symbols())


@pytest.mark.parametrize("mesh", [mi.icosphere(2), mi.split_sphere(4), mi.cube_partition((2, 2, 1), 2),
                                  mi.cut_sphere([0.3, -0.4], 0.35)], ids=lambda m: m.name)
def test_host_tables_match_oracle(lib, mesh):
    h = lib.mtf_mesh_create(mesh.vertices, mesh.triangles, mesh.labels, mesh.n_domains)
    try:
        nd, nt = lib.mtf_mesh_info(h, mesh.n_domains)
        counts = lib.mtf_mesh_pair_counts(h)
    finally:
        lib.mtf_mesh_destroy(h)
    sk = skeleton_of(mesh)
    assert list(nd) == list(sk.N) and nt == sk.n_total
    ref = np.zeros(4, dtype=np.int64)
    for i in range(sk.n_domains):
        pr = classify_pairs(sk, i)
        for c, kname in enumerate(("coincident", "edge", "vertex", "regular")):
            ref[c] += len(pr[kname][0])
    assert list(counts) == list(ref)


def test_reversed_labels_are_canonicalised(lib):
    m = mi.split_sphere(3)
    F = m.triangles.copy()
    L = m.labels.copy()
    F[::2] = F[::2][:, [0, 2, 1]]
    L[::2] = L[::2][:, ::-1]
    h = lib.mtf_mesh_create(m.vertices, F, L, m.n_domains)
    nd, _ = lib.mtf_mesh_info(h, m.n_domains)
    lib.mtf_mesh_destroy(h)
    assert list(nd) == list(skeleton_of(m).N)


def test_invalid_meshes_are_rejected(lib):
    m = mi.split_sphere(3)
    bad = m.labels.copy()
    bad[0] = [2, 2]
    with pytest.raises(lib.MtfError) as e:
        lib.mtf_mesh_create(m.vertices, m.triangles, bad, 3)
    assert e.value.status == 2
    # an open surface: drop one triangle
    with pytest.raises(lib.MtfError) as e:
        lib.mtf_mesh_create(m.vertices, m.triangles[1:], m.labels[1:], 3)
    assert e.value.status == 2
    with pytest.raises(lib.MtfError) as e:
        lib.mtf_mesh_create(m.vertices, m.triangles, m.labels, 1)
    assert e.value.status == 1


def test_default_options(lib):
    """Defaults of the solver options as include/mtf.h documents them; the
    ctypes mirror of mtf_options reads every field of the C struct."""
    from paper_2502_10907_gb300 import _lib as L
    o = L.mtf_default_options()
    assert (o.precision, o.n_ss, o.precond) == (0, 4, 0)
    assert (o.osrc_np, o.max_refine, o.learned) == (4, 4, 0)
    assert (o.osrc_half, o.recycle, o.residual_df) == (1, 1, 1)
    assert o.tol > 0 and o.restart > 0 and o.max_iter > 0
    assert abs(o.osrc_theta - np.pi / 2) < 1e-12 and abs(o.osrc_eps_scale - 0.39) < 1e-12
