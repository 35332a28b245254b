"""Concentric-cuboid meshes (the scatterer of the paper's Sec. 5.4 divided
into M square rings): geometry, orientation and skeleton checks on the CPU."""
import numpy as np
import pytest

import mtf_inputs as mi
from oracle.skeleton import Skeleton


def _domain_of(p, radii):
    """Subdomain of a point from the definition: 0 outside the scatterer, else
    the ring r_{i-1} < max(|x|, |y|) < r_i."""
    w = radii[-1]
    if not (abs(p[0]) < w and abs(p[1]) < w and 0.0 < p[2] < 1.0):
        return 0
    m = max(abs(p[0]), abs(p[1]))
    return 1 + int(np.searchsorted(np.asarray(radii[1:-1]), m))


@pytest.mark.parametrize("M", [1, 2, 3, 6])
def test_cuboid_labels_follow_the_normals(M):
    cfg = mi.config_concentric_cuboids(M, h=0.4)
    m, radii = cfg["mesh"], mi.cuboid_radii(M)
    assert m.n_domains == M + 1
    V, F = m.vertices, m.triangles
    c = V[F].mean(axis=1)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    n /= np.linalg.norm(n, axis=1)[:, None]
    eps = 1e-3
    for t in range(m.nt):
        a, b = m.labels[t]
        assert a < b
        assert _domain_of(c[t] - eps * n[t], radii) == a
        assert _domain_of(c[t] + eps * n[t], radii) == b


@pytest.mark.parametrize("M", [2, 4])
def test_cuboid_subdomain_surfaces_are_closed(M):
    m = mi.config_concentric_cuboids(M, h=0.4)["mesh"]
    for i in range(M + 1):
        sel = np.where((m.labels[:, 0] == i) | (m.labels[:, 1] == i))[0]
        edges = {}
        for t in sel:
            tri = m.triangles[t]
            for k in range(3):
                e = tuple(sorted((int(tri[k]), int(tri[(k + 1) % 3]))))
                edges[e] = edges.get(e, 0) + 1
        assert set(edges.values()) == {2}, i


def test_cuboid_area_and_size():
    # areas of every interface against the geometry; M = 1 at h = 0.18
    # (the size used for the study) has 2,356 triangles and 14,136 unknowns
    M = 3
    m, r = mi.config_concentric_cuboids(M, h=0.3)["mesh"], mi.cuboid_radii(M)
    V, F = m.vertices, m.triangles
    area = 0.5 * np.linalg.norm(np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]]), axis=1)
    for i in range(1, M + 1):
        top_bottom = 2 * ((2 * r[i]) ** 2 - (2 * r[i - 1]) ** 2)
        sel = (m.labels[:, 0] == 0) & (m.labels[:, 1] == i)
        outer = 4 * 2 * r[i] if i == M else 0.0
        assert area[sel].sum() == pytest.approx(top_bottom + outer, rel=1e-12)
        if i < M:
            wall = (m.labels[:, 0] == i) & (m.labels[:, 1] == i + 1)
            assert area[wall].sum() == pytest.approx(4 * 2 * r[i], rel=1e-12)
    m1 = mi.config_concentric_cuboids(1, h=0.18)["mesh"]
    assert m1.nt == 2356
    sk = Skeleton(m1.vertices, m1.triangles, m1.labels, m1.n_domains)
    assert sk.n_total == 14136
