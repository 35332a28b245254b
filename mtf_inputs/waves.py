"""Plane-wave incidences E_inc = p exp(i k0 d.x) (Eq. 22 of the paper's
numerical section), generated deterministically.  Inputs only."""
from __future__ import annotations

import math

import numpy as np


def fibonacci_directions(n: int) -> np.ndarray:
    """n nearly uniform unit vectors on the sphere (Fibonacci lattice)."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def orthonormal_polarizations(d: np.ndarray):
    """Two real unit polarisations orthogonal to each direction d (n, 3)."""
    d = np.asarray(d, dtype=np.float64)
    ref = np.where(np.abs(d[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    p1 = np.cross(ref, d)
    p1 /= np.linalg.norm(p1, axis=1, keepdims=True)
    p2 = np.cross(d, p1)
    return p1, p2


def plane_wave_batch(n_dirs: int):
    """n_dirs Fibonacci directions x 2 orthogonal polarisations -> (2 n_dirs) waves."""
    d = fibonacci_directions(n_dirs)
    p1, p2 = orthonormal_polarizations(d)
    dirs = np.concatenate([d, d])
    pols = np.concatenate([p1, p2]).astype(np.complex128)
    return dirs, pols
