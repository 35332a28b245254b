"""Deterministic synthetic skeleton meshes (inputs only, no method arithmetic).

Every generator returns a :class:`Mesh` whose triangles are oriented so that
the geometric normal points from ``labels[t, 0]`` into ``labels[t, 1]`` with
``labels[t, 0] < labels[t, 1]`` (skeleton orientation of Sec. 3.2 of the
paper: every interface Gamma_ij is meshed once, normal from min(i, j) to
max(i, j)).  Meshes are conforming: interfaces that meet along a curve share
its vertices and edges, which is what lets junction ("triple point") edges
exist (Fig. 1, Table 2 of the paper).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Mesh:
    vertices: np.ndarray   # (nv, 3) float64
    triangles: np.ndarray  # (nt, 3) int32
    labels: np.ndarray     # (nt, 2) int32, labels[t] = (a, b), a < b
    n_domains: int         # M + 1 (the exterior counts)
    name: str = ""

    @property
    def nt(self) -> int:
        return int(self.triangles.shape[0])

    @property
    def nv(self) -> int:
        return int(self.vertices.shape[0])

    def copy(self) -> "Mesh":
        return Mesh(self.vertices.copy(), self.triangles.copy(), self.labels.copy(),
                    self.n_domains, self.name)


# ----------------------------------------------------------------------------
# small helpers
# ----------------------------------------------------------------------------
def _orient(V, F, want):
    """Flip triangles whose normal has a negative component along ``want``.

    ``want`` is an (nt, 3) array of reference directions.
    """
    F = F.copy()
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, want) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


class _VertexPool:
    """Vertex store that deduplicates points by an integer key."""

    def __init__(self):
        self.key2id = {}
        self.pts = []

    def get(self, key, xyz):
        vid = self.key2id.get(key)
        if vid is None:
            vid = len(self.pts)
            self.key2id[key] = vid
            self.pts.append(np.asarray(xyz, dtype=np.float64))
        return vid

    def array(self):
        return np.array(self.pts, dtype=np.float64).reshape(-1, 3)


def _zip_rings(inner, inner_ang, outer, outer_ang):
    """Triangulate the band between two closed rings of vertex ids.

    ``inner`` may be a single vertex (a pole or a disk centre); the band is
    then a fan.  Angles are in [0, 2*pi) and increasing.
    """
    tris = []
    m1, m2 = len(inner), len(outer)
    if m1 == 1:
        for j in range(m2):
            tris.append((inner[0], outer[j], outer[(j + 1) % m2]))
        return tris
    if m2 == 1:
        for i in range(m1):
            tris.append((outer[0], inner[(i + 1) % m1], inner[i]))
        return tris
    a1 = np.concatenate([inner_ang, [inner_ang[0] + 2 * np.pi]])
    a2 = np.concatenate([outer_ang, [outer_ang[0] + 2 * np.pi]])
    i = j = 0
    while i < m1 or j < m2:
        adv_inner = j >= m2 or (i < m1 and a1[i + 1] <= a2[j + 1])
        if adv_inner:
            tris.append((inner[i % m1], inner[(i + 1) % m1], outer[j % m2]))
            i += 1
        else:
            tris.append((inner[i % m1], outer[(j + 1) % m2], outer[j % m2]))
            j += 1
    return tris


# ----------------------------------------------------------------------------
# icosphere
# ----------------------------------------------------------------------------
def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    V = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            V += [(0, s1, s2 * p), (s1, s2 * p, 0), (s2 * p, 0, s1)]
    V = np.array(V, dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    # faces = triples whose plane leaves every other vertex on one side
    faces = []
    n = len(V)
    for a in range(n):
        for b in range(a + 1, n):
            for c in range(b + 1, n):
                nrm = np.cross(V[b] - V[a], V[c] - V[a])
                s = (V - V[a]) @ nrm
                s[[a, b, c]] = 0.0
                if np.all(s <= 1e-12) or np.all(s >= -1e-12):
                    faces.append((a, b, c))
    F = np.array(faces, dtype=np.int64)
    assert F.shape == (20, 3)
    return V, _orient(V, F, V[F].mean(axis=1))


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0),
              inside_label: int = 1) -> Mesh:
    """Sphere = icosahedron refined ``level`` times (20 * 4**level triangles).

    Labels (0, inside_label); the normal points from the exterior (0) into the
    sphere, i.e. inward.
    """
    V, F = _icosahedron()
    V = list(V)
    F = [tuple(f) for f in F]
    for _ in range(level):
        mid = {}
        newF = []

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                mid[key] = len(V) - 1
            return mid[key]

        for (a, b, c) in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            newF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = newF
    V = np.array(V) * radius + np.asarray(center, dtype=np.float64)
    F = np.array(F, dtype=np.int64)
    cen = V[F].mean(axis=1) - np.asarray(center)
    F = _orient(V, F, -cen)  # inward: from exterior 0 into the sphere
    labels = np.tile(np.array([0, inside_label], dtype=np.int32), (len(F), 1))
    return Mesh(V, F.astype(np.int32), labels, inside_label + 1, f"icosphere{level}")


def uv_sphere(rings: int, segments: int, radius: float = 1.0, inside_label: int = 1) -> Mesh:
    """Latitude-longitude sphere: two poles and rings - 1 parallels of
    `segments` points; V = 2 + (rings - 1) segments, so an odd V (and then an
    odd edge count E = 3V - 6) is available, unlike the icosphere family.
    Labels and orientation as icosphere (normal into the sphere)."""
    V = [np.array([0.0, 0.0, 1.0])]
    for r in range(1, rings):
        th = np.pi * r / rings
        for k in range(segments):
            ph = 2 * np.pi * k / segments + 0.5 * r  # twist rings to avoid slivers
            V.append(np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)]))
    V.append(np.array([0.0, 0.0, -1.0]))
    V = np.array(V) * radius
    F = []
    ring = lambda r, k: 1 + (r - 1) * segments + (k % segments)
    for k in range(segments):
        F.append((0, ring(1, k), ring(1, k + 1)))
    for r in range(1, rings - 1):
        for k in range(segments):
            a, b, c, d = ring(r, k), ring(r, k + 1), ring(r + 1, k), ring(r + 1, k + 1)
            F += [(a, c, b), (b, c, d)]
    south = len(V) - 1
    for k in range(segments):
        F.append((south, ring(rings - 1, k + 1), ring(rings - 1, k)))
    F = np.array(F, dtype=np.int64)
    cen = V[F].mean(axis=1)
    F = _orient(V, F, -cen)
    labels = np.tile(np.array([0, inside_label], dtype=np.int32), (len(F), 1))
    return Mesh(V, F.astype(np.int32), labels, inside_label + 1, f"uv_sphere{rings}x{segments}")


# ----------------------------------------------------------------------------
# spheres cut by parallel planes (slab subdomains), rotated at random
# ----------------------------------------------------------------------------
def _disk_rings(pool, z, rho, R, tag):
    """Concentric rings of a disk of radius rho at height z: ring r has 6r
    points (r = 0..R); returns list of (ids, angles)."""
    rings = []
    for r in range(R + 1):
        if r == 0:
            ids = [pool.get((tag, 0, 0), (0.0, 0.0, z))]
            rings.append((ids, np.zeros(1)))
            continue
        m = 6 * r
        ang = 2 * np.pi * np.arange(m) / m
        ids = []
        for k in range(m):
            if r == R:
                key = ("cut", tag, k)  # shared with the sphere ring
            else:
                key = (tag, r, k)
            ids.append(pool.get(key, (rho * r / R * math.cos(ang[k]),
                                      rho * r / R * math.sin(ang[k]), z)))
        rings.append((ids, ang))
    return rings


def cut_sphere(cuts, h: float, radius: float = 1.0, rotation=None,
               name: str = "cut_sphere") -> Mesh:
    """Unit sphere cut by the planes z = c (c in ``cuts``) into slabs.

    Slabs are numbered 1..len(cuts)+1 from the top (largest z).  The sphere
    zone of slab j has labels (0, j) (normal inward); the cut disk between slab
    j and j+1 has labels (j, j+1) (normal pointing down, from j into j+1).
    Latitude rings are spaced about ``h`` apart; each cut disk is a
    6r-per-ring triangulation whose outer ring is the sphere's ring at that
    height.  ``rotation`` (3x3) is applied to all vertices at the end.
    """
    cuts = sorted((float(c) for c in cuts), reverse=True)
    assert all(-1 < c < 1 for c in cuts)
    pool = _VertexPool()
    cut_theta = [math.acos(c) for c in cuts]
    # latitude list: poles, cut latitudes and fillers
    lat = [0.0]
    marks = [0.0] + cut_theta + [math.pi]
    is_cut = []
    for s in range(len(marks) - 1):
        t0, t1 = marks[s], marks[s + 1]
        nseg = max(1, int(round((t1 - t0) * radius / h)))
        for q in range(1, nseg + 1):
            lat.append(t0 + (t1 - t0) * q / nseg)
    cutset = {round(t, 12) for t in cut_theta}
    rings = []
    for li, th in enumerate(lat):
        if li == 0 or li == len(lat) - 1:
            zz = radius if li == 0 else -radius
            rings.append(([pool.get(("pole", li == 0), (0.0, 0.0, zz))], np.zeros(1), False))
            continue
        sr = math.sin(th)
        iscut = round(th, 12) in cutset
        if iscut:
            R = max(1, int(round(radius * sr / h)))
            m = 6 * R
        else:
            m = max(3, int(round(2 * np.pi * radius * sr / h)))
        ang = 2 * np.pi * np.arange(m) / m
        tag = ("cutring", round(th, 12)) if iscut else ("lat", li)
        ids = []
        for k in range(m):
            key = ("cut", tag, k) if iscut else (tag, k)
            ids.append(pool.get(key, (radius * sr * math.cos(ang[k]),
                                      radius * sr * math.sin(ang[k]),
                                      radius * math.cos(th))))
        rings.append((ids, ang, iscut))
    tris, labs, want = [], [], []
    slab = 1
    for li in range(len(rings) - 1):
        (i1, a1, _), (i2, a2, c2) = rings[li], rings[li + 1]
        band = _zip_rings(i1, a1, i2, a2)
        tris += band
        labs += [(0, slab)] * len(band)
        want += ["in"] * len(band)
        if c2:
            # disk below this ring
            th = lat[li + 1]
            R = len(i2) // 6
            tag = ("cutring", round(th, 12))
            drings = _disk_rings(pool, radius * math.cos(th), radius * math.sin(th), R, tag)
            for r in range(R):
                (d1, b1), (d2, b2) = drings[r], drings[r + 1]
                band = _zip_rings(d1, b1, d2, b2)
                tris += band
                labs += [(slab, slab + 1)] * len(band)
                want += ["down"] * len(band)
            slab += 1
    V = pool.array()
    F = np.array(tris, dtype=np.int64)
    cen = V[F].mean(axis=1)
    ref = np.where(np.array(want)[:, None] == "in", -cen, np.array([0.0, 0.0, -1.0]))
    F = _orient(V, F, ref)
    if rotation is not None:
        V = V @ np.asarray(rotation, dtype=np.float64).T
    return Mesh(V, F.astype(np.int32), np.array(labs, dtype=np.int32), len(cuts) + 2, name)


def split_sphere(rings: int = 11, radius: float = 1.0) -> Mesh:
    """Sphere split by the equatorial disk into an upper (1) and a lower (2)
    half; the disk is Gamma_12 and the equator is a triple-junction curve.

    Each of the three surfaces (upper cap, lower cap, disk) has 6*rings**2
    triangles and the equator has 6*rings vertices.
    """
    pool = _VertexPool()
    tris, labs, want = [], [], []
    R = rings
    for part, sgn in (("up", 1.0), ("down", -1.0)):
        prev = None
        for r in range(R + 1):
            th = (r / R) * (np.pi / 2)
            if r == 0:
                ids = [pool.get((part, 0, 0), (0.0, 0.0, sgn * radius))]
                ang = np.zeros(1)
            else:
                m = 6 * r
                ang = 2 * np.pi * np.arange(m) / m
                ids = []
                for k in range(m):
                    key = ("eq", k) if r == R else (part, r, k)
                    ids.append(pool.get(key, (radius * math.sin(th) * math.cos(ang[k]),
                                              radius * math.sin(th) * math.sin(ang[k]),
                                              sgn * radius * math.cos(th))))
            if prev is not None:
                band = _zip_rings(prev[0], prev[1], ids, ang)
                tris += band
                labs += [(0, 1 if sgn > 0 else 2)] * len(band)
                want += ["in"] * len(band)
            prev = (ids, ang)
    prev = None
    for r in range(R + 1):
        if r == 0:
            ids = [pool.get(("disk", 0, 0), (0.0, 0.0, 0.0))]
            ang = np.zeros(1)
        else:
            m = 6 * r
            ang = 2 * np.pi * np.arange(m) / m
            ids = []
            for k in range(m):
                key = ("eq", k) if r == R else ("disk", r, k)
                ids.append(pool.get(key, (radius * r / R * math.cos(ang[k]),
                                          radius * r / R * math.sin(ang[k]), 0.0)))
        if prev is not None:
            band = _zip_rings(prev[0], prev[1], ids, ang)
            tris += band
            labs += [(1, 2)] * len(band)
            want += ["down"] * len(band)
        prev = (ids, ang)
    V = pool.array()
    F = np.array(tris, dtype=np.int64)
    cen = V[F].mean(axis=1)
    ref = np.where(np.array(want)[:, None] == "in", -cen, np.array([0.0, 0.0, -1.0]))
    F = _orient(V, F, ref)
    return Mesh(V, F.astype(np.int32), np.array(labs, dtype=np.int32), 3, f"split_sphere{R}")


# ----------------------------------------------------------------------------
# boxes partitioned into sub-boxes
# ----------------------------------------------------------------------------
def cube_partition(P=(2, 2, 2), n: int = 9, size=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
                   cell_labels=None, name: str = "") -> Mesh:
    """Box [origin, origin+size] split into P[0] x P[1] x P[2] sub-boxes.

    Each sub-box face is an n x n grid of rectangles, each cut into two
    triangles, so every face carries 2 n**2 triangles.  ``cell_labels``
    (shape P) gives the subdomain number of each sub-box (default
    1 + ix + P0*iy + P0*P1*iz).
    """
    P = tuple(int(p) for p in P)
    if cell_labels is None:
        cell_labels = np.zeros(P, dtype=np.int64)
        for ix in range(P[0]):
            for iy in range(P[1]):
                for iz in range(P[2]):
                    cell_labels[ix, iy, iz] = 1 + ix + P[0] * iy + P[0] * P[1] * iz
    cell_labels = np.asarray(cell_labels)
    L = [P[d] * n for d in range(3)]
    h = [size[d] / L[d] for d in range(3)]
    pool = _VertexPool()

    def vid(ijk):
        return pool.get(tuple(ijk), [origin[d] + ijk[d] * h[d] for d in range(3)])

    tris, labs, want = [], [], []
    for d in range(3):
        e1, e2 = (d + 1) % 3, (d + 2) % 3
        for k in range(0, L[d] + 1, n):
            cb = k // n - 1  # cell index on the negative side
            ca = k // n      # cell index on the positive side
            for i in range(L[e1]):
                for j in range(L[e2]):
                    c1, c2 = i // n, j // n

                    def lab(c):
                        if c < 0 or c >= P[d]:
                            return 0
                        idx = [0, 0, 0]
                        idx[d], idx[e1], idx[e2] = c, c1, c2
                        return int(cell_labels[tuple(idx)])

                    lb, la = lab(cb), lab(ca)
                    if lb == la:
                        continue
                    corners = []
                    for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        ijk = [0, 0, 0]
                        ijk[d], ijk[e1], ijk[e2] = k, i + di, j + dj
                        corners.append(vid(ijk))
                    a, b = min(lb, la), max(lb, la)
                    # normal +e_d points from the negative-side cell to the positive one
                    nd = np.zeros(3)
                    nd[d] = 1.0 if lb == a else -1.0
                    for t in ((corners[0], corners[1], corners[2]), (corners[0], corners[2], corners[3])):
                        tris.append(t)
                        labs.append((a, b))
                        want.append(nd)
    V = pool.array()
    F = _orient(V, np.array(tris, dtype=np.int64), np.array(want))
    nd_ = int(cell_labels.max()) + 1
    return Mesh(V, F.astype(np.int32), np.array(labs, dtype=np.int32), nd_,
                name or f"cube{P[0]}x{P[1]}x{P[2]}n{n}")


def grid_partition(xs, ys, zs, cell_labels, name: str = "") -> Mesh:
    """Box [xs[0], xs[-1]] x [ys[0], ys[-1]] x [zs[0], zs[-1]] on the grid of
    the given (increasing) coordinates; cell_labels[i, j, k] is the subdomain
    of cell (xs[i]..xs[i+1]) x (ys[j]..ys[j+1]) x (zs[k]..zs[k+1]), and the
    space outside the box is subdomain 0.  Every grid face between cells of
    different subdomains becomes two triangles (the rectangle cut along its
    diagonal), so the skeleton is conforming by construction."""
    coords = [np.asarray(xs, dtype=np.float64), np.asarray(ys, dtype=np.float64), np.asarray(zs, dtype=np.float64)]
    cell_labels = np.asarray(cell_labels)
    L = [len(c) - 1 for c in coords]
    assert cell_labels.shape == tuple(L)
    pool = _VertexPool()

    def vid(ijk):
        return pool.get(tuple(ijk), [coords[d][ijk[d]] for d in range(3)])

    tris, labs, want = [], [], []
    for d in range(3):
        e1, e2 = (d + 1) % 3, (d + 2) % 3
        for k in range(L[d] + 1):
            for i in range(L[e1]):
                for j in range(L[e2]):
                    def lab(c):
                        if c < 0 or c >= L[d]:
                            return 0
                        idx = [0, 0, 0]
                        idx[d], idx[e1], idx[e2] = c, i, j
                        return int(cell_labels[tuple(idx)])

                    lb, la = lab(k - 1), lab(k)
                    if lb == la:
                        continue
                    corners = []
                    for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        ijk = [0, 0, 0]
                        ijk[d], ijk[e1], ijk[e2] = k, i + di, j + dj
                        corners.append(vid(ijk))
                    a, b = min(lb, la), max(lb, la)
                    nd = np.zeros(3)
                    nd[d] = 1.0 if lb == a else -1.0  # from subdomain a into b
                    for t in ((corners[0], corners[1], corners[2]), (corners[0], corners[2], corners[3])):
                        tris.append(t)
                        labs.append((a, b))
                        want.append(nd)
    V = pool.array()
    F = _orient(V, np.array(tris, dtype=np.int64), np.array(want))
    return Mesh(V, F.astype(np.int32), np.array(labs, dtype=np.int32), int(cell_labels.max()) + 1, name)


def _graded(breaks, h):
    """Grid coordinates through the given breakpoints, each interval split
    into ceil(length / h) equal pieces."""
    out = [float(breaks[0])]
    for a, b in zip(breaks[:-1], breaks[1:]):
        n = max(1, int(math.ceil((b - a) / h - 1e-9)))
        out.extend(float(a + (b - a) * q / n) for q in range(1, n + 1))
    return np.array(out)


def concentric_cuboids(radii, h: float, half_width: float = 1.7, height: float = 1.0) -> Mesh:
    """The scatterer (-w, w)^2 x (0, height), w = half_width, divided into
    M = len(radii) - 1 concentric cuboids: subdomain i (1..M) is the square
    ring r_{i-1} < max(|x|, |y|) < r_i, 0 < z < height, for the radius vector
    radii = [0, r_1, ..., r_M = w].  Structured grid with breakpoints at +-r_i
    and spacing at most h."""
    r = [float(v) for v in radii]
    assert r[0] == 0.0 and abs(r[-1] - half_width) < 1e-12 and all(b > a for a, b in zip(r[:-1], r[1:]))
    M = len(r) - 1
    breaks = sorted({-v for v in r[1:]} | {v for v in r[1:]})
    xs = _graded(breaks, h)
    zs = _graded([0.0, height], h)
    xc = 0.5 * (xs[:-1] + xs[1:])
    lab = np.zeros((len(xc), len(xc), len(zs) - 1), dtype=np.int64)
    for i, x in enumerate(xc):
        for j, y in enumerate(xc):
            m = max(abs(x), abs(y))
            lab[i, j, :] = 1 + int(np.searchsorted(np.array(r[1:-1]), m))
    assert lab.max() == M
    return grid_partition(xs, xs, zs, lab, name=f"cuboids_M{M}_h{h:g}")


def two_disjoint_cubes(n: int = 2, gap: float = 1.0) -> Mesh:
    """Two unit cubes separated by ``gap`` along x (Table 2, 'dielectric')."""
    A = cube_partition((1, 1, 1), n, origin=(0.0, 0.0, 0.0), cell_labels=np.array([[[1]]]))
    B = cube_partition((1, 1, 1), n, origin=(1.0 + gap, 0.0, 0.0), cell_labels=np.array([[[2]]]))
    V = np.concatenate([A.vertices, B.vertices])
    F = np.concatenate([A.triangles, B.triangles + A.nv])
    L = np.concatenate([A.labels, B.labels])
    return Mesh(V, F.astype(np.int32), L.astype(np.int32), 3, "two_cubes")


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a seeded generator (QR of a Gaussian)."""
    A = rng.standard_normal((3, 3))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q
