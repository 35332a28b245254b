"""Convenience wrappers over the C-ABI: handles with destructors, device
buffers from PyTorch (memory and streams only; all compute runs in libmtf)."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Mesh:
    """Skeleton mesh + subdomain spaces (mtf_mesh_create)."""

    def __init__(self, vertices, triangles, labels, n_domains):
        self.n_domains = int(n_domains)
        self.handle = L.mtf_mesh_create(vertices, triangles, labels, n_domains)
        self.n_dofs, self.n_total = L.mtf_mesh_info(self.handle, self.n_domains)
        self.offsets = np.concatenate([[0], np.cumsum(2 * self.n_dofs)]).astype(np.int64)

    @classmethod
    def from_inputs(cls, mesh):
        return cls(mesh.vertices, mesh.triangles, mesh.labels, mesh.n_domains)

    def pair_counts(self):
        return L.mtf_mesh_pair_counts(self.handle)

    def __del__(self):
        if getattr(self, "handle", None):
            L.mtf_mesh_destroy(self.handle)
            self.handle = None


class System:
    """Assembled MTF operator (mtf_assemble) and its solver."""

    def __init__(self, mesh: Mesh, k0, eps_r, mu_r, **opts):
        self.mesh = mesh
        self.opt = L.mtf_default_options()
        for k, v in opts.items():
            setattr(self.opt, k, v)
        self.k0 = float(k0)
        self.handle = L.mtf_assemble(mesh.handle, k0, eps_r, mu_r, self.opt, _stream())

    def reassemble(self, k0, eps_r, mu_r):
        self.k0 = float(k0)
        L.mtf_reassemble(self.handle, k0, eps_r, mu_r, _stream())

    def block(self, i):
        N = int(self.mesh.n_dofs[i])
        T = torch.empty((N, N), dtype=torch.complex128, device="cuda")
        K = torch.empty((N, N), dtype=torch.complex128, device="cuda")
        L.mtf_get_block(self.handle, i, T, K, _stream())
        return T, K

    def matvec(self, x):
        """x: (nrhs, n_total) complex128 cuda tensor (row c = column c of the C-ABI)."""
        x = x.contiguous()
        y = torch.empty_like(x)
        L.mtf_matvec(self.handle, x, y, x.shape[0], _stream())
        return y

    def precond(self, r):
        r = r.contiguous()
        z = torch.empty_like(r)
        L.mtf_precond_apply(self.handle, r, z, r.shape[0], _stream())
        return z

    def matvec_f32(self, x):
        """FP32 streaming matvec (mixed-precision systems); x: (nrhs, n_total) complex64."""
        x = x.contiguous()
        y = torch.empty_like(x)
        L.mtf_matvec_f32(self.handle, x, y, x.shape[0], _stream())
        return y

    def precond_f32(self, r):
        """FP32 block-OSRC apply; r: (nrhs, n_total) complex64."""
        r = r.contiguous()
        z = torch.empty_like(r)
        L.mtf_precond_apply_f32(self.handle, r, z, r.shape[0], _stream())
        return z

    def rhs(self, dirs, pols):
        b = torch.empty((len(dirs), self.mesh.n_total), dtype=torch.complex128, device="cuda")
        L.mtf_rhs(self.handle, dirs, pols, b, _stream())
        return b

    def solve(self, dirs, pols, raise_on_noconv=True):
        x = torch.empty((len(dirs), self.mesh.n_total), dtype=torch.complex128, device="cuda")
        st, status = L.mtf_solve(self.handle, dirs, pols, x, _stream(), raise_on_noconv)
        return x, st

    def farfield(self, x, obs):
        nrhs = x.shape[0]
        f = torch.empty((nrhs, len(obs), 3), dtype=torch.complex128, device="cuda")
        L.mtf_farfield(self.handle, x.contiguous(), nrhs, obs, f, _stream())
        return f

    def __del__(self):
        if getattr(self, "handle", None):
            L.mtf_system_destroy(self.handle)
            self.handle = None
