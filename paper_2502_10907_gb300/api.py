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

    # --- learned correction of block-OSRC (see include/mtf.h) ---------------
    def learned_init(self, kind="table", seed=0):
        """kind: "table" (per-dof stencil coefficients) or "network" (geometry network)."""
        L.mtf_learned_init(self.handle, kind, seed)

    @property
    def learned_param_count(self):
        return L.mtf_learned_param_count(self.handle)

    @property
    def learned_params(self):
        return L.mtf_learned_get_params(self.handle)

    @learned_params.setter
    def learned_params(self, p):
        L.mtf_learned_set_params(self.handle, p)

    def learned_features(self):
        """Geometric features (10, n_dofs) float32 of every dof."""
        x = torch.empty((10, self.mesh.n_total // 2), dtype=torch.float32, device="cuda")
        L.mtf_learned_features(self.handle, x, _stream())
        return x

    def learned_loss_grad(self, x, t, w):
        """Network kind: x (10, rows), t (80, rows), w (rows,) float32 -> (loss, grad)."""
        x, t, w = x.contiguous(), t.contiguous(), w.contiguous()
        g = torch.empty(self.learned_param_count, dtype=torch.float32, device="cuda")
        loss = L.mtf_learned_loss_grad(self.handle, x, t, w, x.shape[1], g, _stream())
        return loss, g

    def learned_power_grad(self, z, c0, K):
        """z (ncols, n_total) complex64 -> (loss, grad) of the K-step power loss with centre c0."""
        z = z.contiguous()
        g = torch.empty(self.learned_param_count, dtype=torch.float32, device="cuda")
        loss = L.mtf_learned_power_grad(self.handle, z, z.shape[0], c0, K, g, _stream())
        return loss, g

    def learned_stencil_adjoint(self, w):
        """w (nrhs, n_total) complex64 -> (C_r^H w, C_P^H w)."""
        w = w.contiguous()
        out_r, out_p = torch.empty_like(w), torch.empty_like(w)
        L.mtf_learned_stencil_adjoint(self.handle, w, out_r, out_p, w.shape[0], _stream())
        return out_r, out_p

    def precond_adjoint_f32(self, w):
        """P^H w for complex64 (nrhs, n_total) w (mixed-precision systems)."""
        w = w.contiguous()
        z = torch.empty_like(w)
        L.mtf_precond_adjoint_f32(self.handle, w, z, w.shape[0], _stream())
        return z

    @property
    def learned_centre(self):
        return L.mtf_learned_centre(self.handle)

    def learned_train(self, steps, lr=3e-3, batch=16, K=6, seed=0):
        return L.mtf_learned_train(self.handle, steps, lr, batch, K, seed, _stream())

    def learned_fit(self, dirs, pols, rounds=4, steps_per_round=150, lr=3e-3, batch=16, K=6, seed=0):
        """Train with validation on the plane waves (dirs, pols); returns the report as a dict."""
        return L.mtf_learned_fit(self.handle, dirs, pols, rounds, steps_per_round, lr, batch, K, seed, _stream())

    def learned_enable(self, on=True):
        L.mtf_learned_enable(self.handle, on)

    def learned_apply(self, r):
        r = r.contiguous()
        z = torch.empty_like(r)
        L.mtf_learned_apply(self.handle, r, z, r.shape[0], _stream())
        return z

    def matvec_f32(self, x):
        """FP32 streaming matvec (mixed-precision systems); x: (nrhs, n_total) complex64."""
        x = x.contiguous()
        y = torch.empty_like(x)
        L.mtf_matvec_f32(self.handle, x, y, x.shape[0], _stream())
        return y

    def matvec_adjoint_f32(self, v):
        """M^H v (mixed-precision systems); v: (nrhs, n_total) complex64."""
        v = v.contiguous()
        y = torch.empty_like(v)
        L.mtf_matvec_adjoint_f32(self.handle, v, y, v.shape[0], _stream())
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

    def autotune(self, nrhs, reps=5):
        """Time the operator-apply plans for nrhs right-hand sides and keep the fastest (report lines)."""
        return L.mtf_autotune(self.handle, nrhs, reps, _stream())

    def solve_rhs(self, b, raise_on_noconv=True):
        """Solve M x = b for b (nrhs, n_total) complex128 on the GPU."""
        b = b.contiguous()
        x = torch.empty_like(b)
        st, status = L.mtf_solve_rhs(self.handle, b, x, _stream(), raise_on_noconv)
        return x, st

    def nearfield(self, x, points, domains):
        """U at points (P, 3) in subdomains domains (P,) by Eq. 8 -> (nrhs, P, 3) complex128:
        the scattered field in subdomain 0, the total field in the others."""
        x = x.contiguous()
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        f = torch.empty((x.shape[0], len(pts), 3), dtype=torch.complex128, device="cuda")
        L.mtf_nearfield(self.handle, x, x.shape[0], pts, domains, f, _stream())
        return f

    def farfield(self, x, obs):
        nrhs = x.shape[0]
        f = torch.empty((nrhs, len(obs), 3), dtype=torch.complex128, device="cuda")
        L.mtf_farfield(self.handle, x.contiguous(), nrhs, obs, f, _stream())
        return f

    def __del__(self):
        if getattr(self, "handle", None):
            L.mtf_system_destroy(self.handle)
            self.handle = None


def solve_batch(systems, dirs_list, pols_list, threads=0, raise_on_noconv=True):
    """Solve independent instances together (mtf_solve_batch): one (nrhs_i, n_total_i)
    complex128 solution per system, and the per-instance stats."""
    xs = [torch.empty((len(d), s.mesh.n_total), dtype=torch.complex128, device="cuda")
          for s, d in zip(systems, dirs_list)]
    st, status = L.mtf_solve_batch([s.handle for s in systems], dirs_list, pols_list, xs, threads, _stream(),
                                   raise_on_noconv)
    return xs, st
