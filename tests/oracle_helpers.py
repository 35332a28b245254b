"""Shared helpers for the oracle tests (test-side only)."""
import numpy as np

import mtf_inputs as mi
from oracle.skeleton import Skeleton
from oracle.mtf import MTFSystem


def skeleton_of(mesh):
    return Skeleton(mesh.vertices, mesh.triangles, mesh.labels, mesh.n_domains)


def sphere_system(cache, level, k0=1.0, eps=2.0):
    key = ("sphere", level, k0, eps)
    if key not in cache:
        cfg = mi.config_sphere(level=level, k0=k0, eps=eps)
        sk = skeleton_of(cfg["mesh"])
        cache[key] = (cfg, sk, MTFSystem(sk, cfg["k0"], cfg["eps_r"], cfg["mu_r"]))
    return cache[key]


def rcs_plane(n=91):
    th = np.linspace(0.0, np.pi, n)
    return np.stack([np.cos(th), np.sin(th), 0.0 * th], axis=1)
