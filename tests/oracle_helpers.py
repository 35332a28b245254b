"""Shared helpers for the oracle tests (test-side only)."""
import numpy as np

import mtf_inputs as mi
from oracle.skeleton import Skeleton
from oracle.mtf import MTFSystem
from oracle.operators import triangle_points, _rwg_data


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


def jump_l2(sk, x, i, j):
    """Relative L2 norm over Gamma_ij of the Dirichlet and Neumann jumps
    u_i + u_j (the transmission conditions make the fields opposite)."""
    lo, hi = min(i, j), max(i, j)
    tris = np.where((sk.L[:, 0] == lo) & (sk.L[:, 1] == hi))[0]
    X, W = triangle_points(sk, tris)
    out = []
    for slot in (0, 1):
        fields = []
        for dom in (i, j):
            pos = {t: p for p, t in enumerate(sk.tris[dom])}
            loc = np.array([pos[t] for t in tris])
            c, v = _rwg_data(sk, dom, loc)
            sl = sk.block_slices(dom)[slot]
            coef = x[sl, 0][sk.dof[dom][loc]]
            f = c[:, :, None, None] * (X[:, None] - v[:, :, None, :])
            fields.append(np.einsum("ta,taqn->tqn", coef, f))
        jump = fields[0] + fields[1]
        nrm = lambda u: np.sqrt(np.sum(W * np.sum(np.abs(u) ** 2, axis=-1)))
        out.append(nrm(jump) / nrm(fields[0]))
    return out
