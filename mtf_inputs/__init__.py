"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package only *generates inputs*: skeleton meshes (vertices, triangles,
subdomain labels), material parameters and plane-wave incidences.  It holds
none of the arithmetic of the method (no quadrature, no operators, no
solver), so that the CPU oracle and the CUDA library can both be fed from it
while sharing no code with each other.

Label convention of every mesh produced here: ``labels[t] = (a, b)`` with
``a < b`` and the geometric normal of triangle ``t`` (right-hand rule on its
vertex order) pointing from subdomain ``a`` into subdomain ``b``; subdomain 0
is the unbounded exterior.  This is the "normal from min(i,j) to max(i,j)"
orientation of the skeleton mesh described in Sec. 3.2 of the paper.
"""
from .meshes import (icosphere, uv_sphere, split_sphere, cube_partition, two_disjoint_cubes,
                     cut_sphere, grid_partition, concentric_cuboids, Mesh)
from .waves import fibonacci_directions, orthonormal_polarizations, plane_wave_batch
from .configs import (config_sphere, config_split_sphere, config_cube2,
                      config_cube4, config_batch_instances, config_concentric_cuboids, cuboid_radii,
                      CONFIG_NAMES)

__all__ = [
    "Mesh", "icosphere", "uv_sphere", "split_sphere", "cube_partition", "two_disjoint_cubes",
    "cut_sphere", "grid_partition", "concentric_cuboids", "fibonacci_directions", "orthonormal_polarizations",
    "plane_wave_batch", "config_sphere", "config_split_sphere", "config_cube2",
    "config_cube4", "config_batch_instances", "config_concentric_cuboids", "cuboid_radii",
    "CONFIG_NAMES",
]
