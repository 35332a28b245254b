"""The MTF linear system, its solution and the far field (oracle side).

Problem 2 of the paper: M = 2A + X with A = diag(A_i),

    A_i = [[K_i, rho_i^-1 T_i], [-rho_i T_i, K_i]]        (Eq. 9, scaled Calderon)

at wavenumber k_i = k0 sqrt(eps_r,i mu_r,i), rho_i = sqrt(eps_r,i / mu_r,i)
(Eq. 1), and X the transmission couplings I_ji of Eq. (11)-(13), which act
with the same sign on both traces (Remark 2).

Unknowns of block i (Eq. 14): u_i = (gamma_D E, rho_i gamma_N E) expanded in
RWG_i x RWG_i; the global vector stacks blocks i = 0..M, each as
[D coefficients (N_i), N coefficients (N_i)].  Rows are tested with the
x-pairing against RWG_i in the same slot order (a row permutation of the
slot-swapping pairing of Eq. 6, which leaves the solution unchanged).

Right-hand side: the projector identity (Eq. 10) holds for every block
(A_i u = u / 2 for Cauchy data of fields solving Maxwell in Omega_i, radiating
if i = 0), while the incident wave, regular inside the scatterer, satisfies
the complementary identity A_0 u_inc = -u_inc / 2 on Gamma_0 (traces taken
with n_0).  Adding the two gives 2 A_0 u_0 - u_0 = -2 u_0^inc, so block 0 of
the right-hand side is -2 times the tested incident traces and all other
blocks are zero.  (Proposition 1 of the paper writes +2 u_inc; its appendix
derivation flips the sign of Eq. (10) for Omega_0.  The reading here is the
one the projector identities give, and the Mie series pins it.)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .skeleton import Skeleton
from .operators import (assemble_block, transmission_gram, incident_data,
                        triangle_points, _rwg_data)


def material(k0, eps_r, mu_r):
    """k_i = k0 sqrt(eps_r mu_r) and rho_i = sqrt(eps_r / mu_r)  (Eq. 1)."""
    eps_r = np.asarray(eps_r, dtype=np.complex128)
    mu_r = np.asarray(mu_r, dtype=np.complex128)
    return k0 * np.sqrt(eps_r * mu_r), np.sqrt(eps_r / mu_r)


class MTFSystem:
    """Dense FP64 MTF matrix of Problem 2 for a skeleton mesh."""

    def __init__(self, sk: Skeleton, k0, eps_r, mu_r, n_ss: int = 4, assemble: bool = True):
        self.sk = sk
        self.k0 = float(k0)
        self.k, self.rho = material(k0, eps_r, mu_r)
        self.n_ss = n_ss
        self.T, self.K = [], []
        if assemble:
            for i in range(sk.n_domains):
                Ti, Ki = assemble_block(sk, i, self.k[i], n_ss=n_ss)
                self.T.append(Ti)
                self.K.append(Ki)
        self.G = {}
        for i in range(sk.n_domains):
            for j in sk.Lambda[i]:
                self.G[(i, j)] = transmission_gram(sk, i, j)

    # ------------------------------------------------------------------
    def calderon_block(self, i):
        """Galerkin matrix of the scaled Calderon operator A_i (2N_i x 2N_i)."""
        T, K, r = self.T[i], self.K[i], self.rho[i]
        return np.block([[K, T / r], [-r * T, K]])

    def matrix(self):
        """Dense M = 2A + X (n_total x n_total)."""
        sk = self.sk
        M = np.zeros((sk.n_total, sk.n_total), dtype=np.complex128)
        for i in range(sk.n_domains):
            o = sk.offset[i]
            n2 = 2 * sk.N[i]
            M[o:o + n2, o:o + n2] = 2.0 * self.calderon_block(i)
            Di, Ni = sk.block_slices(i)
            for j in sk.Lambda[i]:
                Dj, Nj = sk.block_slices(j)
                M[Di, Dj] += self.G[(i, j)]
                M[Ni, Nj] += self.G[(i, j)]
        return M

    def matvec(self, x):
        """y = M x computed block by block (same result as matrix() @ x)."""
        sk = self.sk
        x = np.asarray(x)
        y = np.zeros_like(x, dtype=np.complex128)
        for i in range(sk.n_domains):
            Di, Ni = sk.block_slices(i)
            r = self.rho[i]
            y[Di] = 2.0 * (self.K[i] @ x[Di] + (self.T[i] @ x[Ni]) / r)
            y[Ni] = 2.0 * (-r * (self.T[i] @ x[Di]) + self.K[i] @ x[Ni])
            for j in sk.Lambda[i]:
                Dj, Nj = sk.block_slices(j)
                y[Di] += self.G[(i, j)] @ x[Dj]
                y[Ni] += self.G[(i, j)] @ x[Nj]
        return y

    def rhs(self, dirs, pols):
        """Right-hand sides (n_total, nrhs): block 0 = -2 (tested incident traces)."""
        sk = self.sk
        dirs = np.atleast_2d(dirs)
        pols = np.atleast_2d(pols)
        b = np.zeros((sk.n_total, len(dirs)), dtype=np.complex128)
        D0, N0 = sk.block_slices(0)
        for c, (d, p) in enumerate(zip(dirs, pols)):
            bD, bN = incident_data(sk, self.k0, d, p)
            b[D0, c] = -2.0 * bD
            b[N0, c] = -2.0 * bN
        return b

    def solve_lu(self, b):
        """Direct LU solve (the small-case solver of Sec. 5.2)."""
        lu = scipy.linalg.lu_factor(self.matrix())
        return scipy.linalg.lu_solve(lu, b)

    # ------------------------------------------------------------------
    def farfield(self, x, obs):
        """Far field E_inf(xhat) of the solution(s) x at unit directions obs.

        From the Stratton-Chu representation (Eq. 8) in Omega_0 with the total
        Cauchy data u_0 (the incident part radiates nothing into Omega_0):
        E_sc = H(a) + E(b), a = gamma_D E, b = gamma_N E on Gamma_0 (rho_0 = 1).
        With E_sc(x) ~ exp(i k0 |x|) / |x| E_inf(xhat):
        E_inf = i k0 / (4 pi) [xhat x w_a + (xhat x w_b) x xhat],
        w_. = int_{Gamma_0} (trace)(y) exp(-i k0 xhat . y) dy.
        Returns (n_obs, 3, nrhs) complex.
        """
        sk = self.sk
        x = np.atleast_2d(np.asarray(x).T).T
        obs = np.atleast_2d(obs)
        D0, N0 = sk.block_slices(0)
        loc = np.arange(len(sk.tris[0]))
        c, v = _rwg_data(sk, 0, loc)
        X, W = triangle_points(sk, sk.tris[0])                      # (T,Q,3)
        f = c[:, :, None, None] * (X[:, None] - v[:, :, None, :])    # (T,3,Q,3)
        dof = sk.dof[0]
        out = np.zeros((len(obs), 3, x.shape[1]), dtype=np.complex128)
        phase = np.exp(-1j * self.k0 * np.einsum("tqn,on->otq", X, obs))   # (O,T,Q)
        for r in range(x.shape[1]):
            a_cf = x[D0, r][dof]   # (T,3)
            b_cf = x[N0, r][dof]
            a = np.einsum("ta,taqn->tqn", a_cf, f)
            b = np.einsum("ta,taqn->tqn", b_cf, f)
            wa = np.einsum("otq,tq,tqn->on", phase, W, a)
            wb = np.einsum("otq,tq,tqn->on", phase, W, b)
            out[:, :, r] = (1j * self.k0 / (4 * np.pi)) * (
                np.cross(obs, wa) + np.cross(np.cross(obs, wb), obs))
        return out
