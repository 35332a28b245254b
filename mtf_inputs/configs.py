"""The five synthetic workloads (meshes, materials, incidences) used by the
tests and the benchmark.  All draws are seeded (numpy PCG64).

Each function returns a dict with keys ``mesh`` (a :class:`Mesh`), ``k0``,
``eps_r`` and ``mu_r`` (length n_domains, index 0 = vacuum), ``dirs``
(nrhs, 3) and ``pols`` (nrhs, 3) complex.
"""
from __future__ import annotations

import numpy as np

from .meshes import icosphere, split_sphere, cube_partition, cut_sphere, random_rotation, concentric_cuboids
from .waves import plane_wave_batch

CONFIG_NAMES = ("sphere", "split_sphere", "cube2", "batch_instances", "cube4")


def config_sphere(level: int = 2, k0: float = 1.0, eps: float = 2.0):
    """Dielectric sphere radius 1 (eps_r=2, mu_r=1) in vacuum, k0=1, icosphere
    level 2 (320 triangles, 480 edges), one x-polarised wave along +z."""
    mesh = icosphere(level)
    return dict(name=f"sphere_L{level}", mesh=mesh, k0=k0,
                eps_r=np.array([1.0, eps]), mu_r=np.array([1.0, 1.0]),
                dirs=np.array([[0.0, 0.0, 1.0]]),
                pols=np.array([[1.0, 0.0, 0.0]], dtype=np.complex128))


def config_split_sphere(rings: int = 11, k0: float = 2.0):
    """Sphere radius 1 split into two hemispheres by the equator disk (three
    subdomains with a triple-junction equator), eps_r = 2 (upper) and 4
    (lower), k0 = 2, 6*rings**2 triangles per surface, two polarisations of a
    wave along +z."""
    mesh = split_sphere(rings)
    return dict(name=f"split_sphere_R{rings}", mesh=mesh, k0=k0,
                eps_r=np.array([1.0, 2.0, 4.0]), mu_r=np.ones(3),
                dirs=np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]]),
                pols=np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], dtype=np.complex128))


def config_cube2(n: int = 9, k0: float = 3.0, n_dirs: int = 32, seed: int = 0):
    """Unit cube partitioned 2x2x2, eps_r i.i.d. U[1.5, 4], mu_r = 1, k0 = 3,
    2*n**2 triangles per square face, n_dirs Fibonacci directions x 2
    polarisations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = cube_partition((2, 2, 2), n)
    eps = np.concatenate([[1.0], rng.uniform(1.5, 4.0, mesh.n_domains - 1)])
    dirs, pols = plane_wave_batch(n_dirs)
    return dict(name=f"cube2_n{n}", mesh=mesh, k0=k0, eps_r=eps,
                mu_r=np.ones(mesh.n_domains), dirs=dirs, pols=pols)


def config_cube4(n: int = 5, k0: float = 4.0, n_dirs: int = 8, seed: int = 0):
    """Unit cube partitioned 4x4x4, eps_r U[1.5, 6], k0 = 4, 2*n**2 triangles
    per face, 2*n_dirs right-hand sides."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = cube_partition((4, 4, 4), n)
    eps = np.concatenate([[1.0], rng.uniform(1.5, 6.0, mesh.n_domains - 1)])
    dirs, pols = plane_wave_batch(n_dirs)
    return dict(name=f"cube4_n{n}", mesh=mesh, k0=k0, eps_r=eps,
                mu_r=np.ones(mesh.n_domains), dirs=dirs, pols=pols)


def config_batch_instances(n_inst: int = 32, seed: int = 0, tri_range=(500, 5000),
                           nrhs: int = 8):
    """Uneven instances: unit spheres cut by 1..15 parallel planes at random
    heights (2..16 slab subdomains), rotated at random, 500-5000 triangles,
    k0 ~ U[1, 4], eps_r ~ U[1.5, 6], nrhs waves each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(n_inst):
        ncut = int(rng.integers(1, 16))
        target = float(rng.uniform(*tri_range))
        cuts = np.sort(rng.uniform(-0.85, 0.85, ncut))
        # keep cuts apart so that slabs are not degenerate
        cuts = np.linspace(-0.85, 0.85, ncut) * 0.5 + 0.5 * cuts
        rot = random_rotation(rng)
        # sphere + disks area ~ 4 pi + sum pi (1 - c^2); triangles ~ 2.3 area / h^2
        area = 4 * np.pi + np.pi * np.sum(1 - cuts ** 2)
        h = float(np.sqrt(2.3 * area / target))
        mesh = cut_sphere(cuts, h, rotation=rot, name=f"inst{q}")
        k0 = float(rng.uniform(1.0, 4.0))
        eps = np.concatenate([[1.0], rng.uniform(1.5, 6.0, mesh.n_domains - 1)])
        dirs, pols = plane_wave_batch(nrhs // 2)
        out.append(dict(name=f"inst{q}", mesh=mesh, k0=k0, eps_r=eps,
                        mu_r=np.ones(mesh.n_domains), dirs=dirs, pols=pols))
    return out


def cuboid_radii(M: int):
    """Radius vector [0, r_1, ..., r_M = 1.7] of the M concentric cuboids:
    r_1 = 0.5 and the outer radii equally spaced up to 1.7 (M = 2 gives
    [0, 0.5, 1.7]); M = 1 is the undivided scatterer [0, 1.7]."""
    if M == 1:
        return [0.0, 1.7]
    return [0.0] + [float(v) for v in np.linspace(0.5, 1.7, M)]


def config_concentric_cuboids(M: int = 1, h: float = 0.18, k0: float = 3.0, eps: float = 2.0):
    """The scatterer (-1.7, 1.7)^2 x (0, 1) divided into M concentric cuboids
    (square rings), every ring with eps_r = eps and mu_r = 1 (k_i = k0
    sqrt(eps) = 4.24 at the defaults), structured grid of spacing <= h
    (h = 0.18 gives 2,356 skeleton triangles, 14,136 unknowns at M = 1); one
    z-polarised plane wave travelling along +x."""
    mesh = concentric_cuboids(cuboid_radii(M), h)
    return dict(name=f"cuboids_M{M}_h{h:g}", mesh=mesh, k0=k0,
                eps_r=np.array([1.0] + [eps] * M), mu_r=np.ones(M + 1),
                dirs=np.array([[1.0, 0.0, 0.0]]), pols=np.array([[0.0, 0.0, 1.0]], dtype=np.complex128))
