"""Skeleton-mesh bookkeeping (oracle side): Algorithm 1 and RWG tables.

Follows Sec. 4.2 ("Top-down approach for space definitions"), Algorithm 1
("Process subdomains and swap normals") and Table 2 of the paper.

Readings taken where the paper is silent:

* Input triangles may carry labels (a, b) in either order; the triangle is
  re-oriented so that its normal points from min(a, b) to max(a, b), the
  convention Algorithm 1 assumes (Sec. 3.2).
* RWG_i is the standard closed-surface RWG space on Gamma_i (one dof per edge
  of Gamma_i, including junction edges).  Dofs of Gamma_i are numbered by
  increasing (lower vertex id, higher vertex id) of the edge.
* Orientation sign of the RWG function of edge e on triangle t in subdomain i:
  s = dir(e, t) * swap_i(t), where dir = +1 if the triangle's vertex order
  runs along e from the lower to the higher vertex id, else -1.  On a
  consistently oriented closed Gamma_i the two triangles of an edge get
  opposite signs (div-conformity); on a triangle of Gamma_ij the RWG_i and
  RWG_j functions of the same edge are opposite (swap_i = -swap_j).
* RWG function: f(x) = s * l / (2 A) * (x - v), v the vertex opposite e,
  l = |e|, A = area of t; div f = s * l / A.
"""
from __future__ import annotations

import numpy as np


class Skeleton:
    """Subdomain spaces RWG_i and normal multipliers NM_i of a skeleton mesh."""

    def __init__(self, vertices, triangles, labels, n_domains):
        V = np.asarray(vertices, dtype=np.float64)
        F = np.asarray(triangles, dtype=np.int64).copy()
        L = np.asarray(labels, dtype=np.int64).copy()
        if np.any(L[:, 0] == L[:, 1]):
            raise ValueError("a triangle must separate two distinct subdomains")
        flip = L[:, 0] > L[:, 1]
        F[flip] = F[flip][:, [0, 2, 1]]
        L[flip] = L[flip][:, ::-1]
        self.V, self.F, self.L = V, F, L
        self.n_domains = int(n_domains)
        nt = len(F)
        # geometry
        e1 = V[F[:, 1]] - V[F[:, 0]]
        e2 = V[F[:, 2]] - V[F[:, 0]]
        cr = np.cross(e1, e2)
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        self.normal = cr / (2.0 * self.area[:, None])  # from L[:,0] into L[:,1]
        # Lambda_i: neighbour sets (Sec. 2.1)
        self.Lambda = [sorted(set(L[L[:, 0] == i, 1]) | set(L[L[:, 1] == i, 0]))
                       for i in range(self.n_domains)]
        # Algorithm 1: for each i and j in Lambda_i, swap = sign(j - i) and the
        # triangles of Gamma_ij join RWG_i with that swap.
        self.tris = []   # per domain: int array of triangle ids
        self.swap = []   # per domain: +-1 per triangle
        for i in range(self.n_domains):
            ts, sw = [], []
            for j in self.Lambda[i]:
                lo, hi = min(i, j), max(i, j)
                sel = np.where((L[:, 0] == lo) & (L[:, 1] == hi))[0]
                ts.append(sel)
                sw.append(np.full(len(sel), 1 if j > i else -1))
            self.tris.append(np.concatenate(ts) if ts else np.zeros(0, np.int64))
            self.swap.append(np.concatenate(sw) if sw else np.zeros(0, np.int64))
        # per-domain RWG tables
        self.N = []
        self.dof = []     # per domain: (T_i, 3) local dof of the edge opposite vertex a
        self.sign = []    # per domain: (T_i, 3)
        self.length = []  # per domain: (T_i, 3)
        self.edges = []   # per domain: (N_i, 2) vertex pairs of the dofs
        for i in range(self.n_domains):
            t = self.tris[i]
            Ft = F[t]
            ends = np.stack([Ft[:, [1, 2]], Ft[:, [2, 0]], Ft[:, [0, 1]]], axis=1)  # (T,3,2)
            lo = np.minimum(ends[..., 0], ends[..., 1])
            hi = np.maximum(ends[..., 0], ends[..., 1])
            keys = lo * (len(V) + 1) + hi
            uniq, inv = np.unique(keys.ravel(), return_inverse=True)
            self.N.append(len(uniq))
            self.dof.append(inv.reshape(-1, 3))
            direction = np.where(ends[..., 0] < ends[..., 1], 1, -1)
            self.sign.append(direction * self.swap[i][:, None])
            self.length.append(np.linalg.norm(V[ends[..., 1]] - V[ends[..., 0]], axis=2))
            self.edges.append(np.stack([uniq // (len(V) + 1), uniq % (len(V) + 1)], axis=1))
        self.offset = np.concatenate([[0], np.cumsum([2 * n for n in self.N])]).astype(np.int64)
        self.n_total = int(self.offset[-1])

    # ------------------------------------------------------------------
    def signed_interface_list(self, i):
        """Gamma_i as the signed list of Table 2 (e.g. ['-01', '12'])."""
        out = []
        for j in self.Lambda[i]:
            lo, hi = min(i, j), max(i, j)
            out.append(("" if j > i else "-") + f"{lo}{hi}")
        return out

    def rwg_coeff(self, i):
        """c[t, a] = s l / (2 A): RWG f_a(x) = c (x - v_a) on triangle t of Gamma_i."""
        t = self.tris[i]
        return self.sign[i] * self.length[i] / (2.0 * self.area[t][:, None])

    def outward_normal(self, i):
        """n_i on each triangle of Gamma_i (swap * skeleton normal)."""
        return self.swap[i][:, None] * self.normal[self.tris[i]]

    def block_slices(self, i):
        """(D-slot slice, N-slot slice) of block i in the global unknown vector."""
        o, n = int(self.offset[i]), self.N[i]
        return slice(o, o + n), slice(o + n, o + 2 * n)
