"""Block-OSRC preconditioner (oracle side), Sec. 4.4 of the paper.

The paper defines the block preconditioner
    A~_i = [[0, rho_i^-1 T~], [-rho_i T~, 0]]          (Eq. 19)
with T~ = Pi~^{-1}_{k, eps, N_p} an OSRC approximation of the EtM map
EtM = -T^{-1}(I/2 + K), built from a Pade approximation (order N_p, damped
wavenumber k_eps = k + i eps) of a square-root surface operator, and leaves
its discretisation to the cited OSRC work.  Reading taken here (stated in
the design notes; the CUDA library implements the same operator):

* Principal symbols of the Galerkin EFIO on a flat patch: on irrotational
  currents with div-div / mass eigenvalue lambda (= |xi|^2) the EFIO acts as
  i q / (2k), q = sqrt(lambda - k^2) (outgoing branch), on solenoidal ones as
  -i k / (2q); both inverses equal 2k / sqrt(k^2 - lambda) at lambda = 0 and
  the first is the OSRC square-root symbol
      T^{-1} ~ 2k / (k_eps sqrt(1 + Z)),   Z = -lambda / k_eps^2,
  i.e. sqrt(1 + X / k_eps^2) with X = grad_G div_G (the curl-curl part of the
  Hodge Laplacian, which RWG cannot represent conformingly, is dropped).
* sqrt(1 + Z) is replaced by the rotating-branch-cut Pade approximant of
  order N_p and angle theta (Milinazzo, Zala & Brooke 1997):
      a_j = 2/(2N_p+1) sin^2(j pi/(2N_p+1)), b_j = cos^2(j pi/(2N_p+1)),
      R(z) = 1 + sum a_j z / (1 + b_j z),
      sqrt(1+z) ~ C0 + sum A_j z / (1 + B_j z),
      C0 = e^{i theta/2} R(e^{-i theta} - 1),
      A_j = e^{-i theta/2} a_j / (1 + b_j (e^{-i theta} - 1))^2,
      B_j = e^{-i theta} b_j / (1 + b_j (e^{-i theta} - 1)).
* Damping eps = c k^{1/3} R^{-2/3} (c = 0.39, R the radius of the sphere with
  the area of Gamma_i), the curvature-based choice of the OSRC literature.
* Discretisation: with the RWG mass G and div-div matrix D of Gamma_i and the
  generalised eigenpairs D v = lambda G v, V^T G V = I, the operator is
      T~ = V diag(f(lambda)) V^T,  f = 2k / (k_eps P(-lambda / k_eps^2)),
  which maps tested vectors to coefficients (V V^T = G^{-1}); the Pade
  approximant is applied exactly on each eigenvalue instead of through
  auxiliary sparse solves.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .operators import mass_matrix, triangle_points, _rwg_data, _scatter
from .skeleton import Skeleton


def divdiv_matrix(sk: Skeleton, i: int):
    """D[m, n] = int_{Gamma_i} div psi_m div psi_n (piecewise constant divergences)."""
    N = sk.N[i]
    Dm = np.zeros((N, N))
    c = sk.rwg_coeff(i)                      # div psi_a = 2 c_a on each triangle
    area = sk.area[sk.tris[i]]
    loc = area[:, None, None] * (2 * c)[:, :, None] * (2 * c)[:, None, :]
    _scatter(Dm, sk.dof[i], sk.dof[i], loc)
    return Dm


def pade_coefficients(Np: int, theta: float):
    """(C0, A, B) of the rotated-branch-cut Pade approximant of sqrt(1 + z)."""
    j = np.arange(1, Np + 1)
    a = 2.0 / (2 * Np + 1) * np.sin(j * np.pi / (2 * Np + 1)) ** 2
    b = np.cos(j * np.pi / (2 * Np + 1)) ** 2
    e = np.exp(-1j * theta)
    R = 1.0 + np.sum(a * (e - 1.0) / (1.0 + b * (e - 1.0)))
    C0 = np.exp(1j * theta / 2) * R
    A = np.exp(-1j * theta / 2) * a / (1.0 + b * (e - 1.0)) ** 2
    B = e * b / (1.0 + b * (e - 1.0))
    return C0, A, B


def pade_sqrt(z, Np: int = 4, theta: float = np.pi / 2):
    C0, A, B = pade_coefficients(Np, theta)
    z = np.asarray(z, dtype=np.complex128)
    return C0 + np.sum(A[None, :] * z[..., None] / (1.0 + B[None, :] * z[..., None]), axis=-1)


def damping(k, area, scale=0.39):
    R = np.sqrt(area / (4 * np.pi))
    return scale * np.real(k) ** (1.0 / 3.0) * R ** (-2.0 / 3.0)


class BlockOSRC:
    """Block-OSRC preconditioner of an MTF system (Eq. 19)."""

    def __init__(self, sk: Skeleton, k, rho, Np=4, theta=np.pi / 2, eps_scale=0.39):
        self.sk = sk
        self.rho = np.asarray(rho)
        self.Ttil = []
        for i in range(sk.n_domains):
            G = mass_matrix(sk, i)
            D = divdiv_matrix(sk, i)
            lam, V = scipy.linalg.eigh(D, G)
            area = float(np.sum(sk.area[sk.tris[i]]))
            keps = k[i] + 1j * damping(k[i], area, eps_scale)
            f = 2 * k[i] / (keps * pade_sqrt(-lam / keps ** 2, Np, theta))
            self.Ttil.append((V * f[None, :]) @ V.T)

    def apply(self, r):
        """z = A~ r blockwise: z_D = rho^-1 T~ r_N, z_N = -rho T~ r_D."""
        r = np.asarray(r)
        z = np.zeros_like(r, dtype=np.complex128)
        for i in range(self.sk.n_domains):
            Di, Ni = self.sk.block_slices(i)
            z[Di] = (self.Ttil[i] @ r[Ni]) / self.rho[i]
            z[Ni] = -self.rho[i] * (self.Ttil[i] @ r[Di])
        return z

    def matrix(self):
        sk = self.sk
        P = np.zeros((sk.n_total, sk.n_total), dtype=np.complex128)
        for i in range(sk.n_domains):
            Di, Ni = sk.block_slices(i)
            P[Di, Ni] = self.Ttil[i] / self.rho[i]
            P[Ni, Di] = -self.rho[i] * self.Ttil[i]
        return P


def gmres_iterations(A, b, tol, restart, maxit, P=None):
    """Plain right-preconditioned restarted GMRES (CGS2) on dense matrices;
    returns (x, iterations, converged).  Reference for iteration counts."""
    n = len(b)
    x = np.zeros(n, dtype=np.complex128)
    bn = np.linalg.norm(b)
    tot = 0
    AP = A if P is None else A @ P
    while tot < maxit:
        r = b - AP @ x
        beta = np.linalg.norm(r)
        if beta / bn <= tol:
            return (x if P is None else P @ x), tot, True
        V = np.zeros((n, restart + 1), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        V[:, 0] = r / beta
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        for j in range(restart):
            w = AP @ V[:, j]
            for _ in range(2):
                h = V[:, :j + 1].conj().T @ w
                w = w - V[:, :j + 1] @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / H[j + 1, j]
            tot += 1
            y = np.linalg.lstsq(H[:j + 2, :j + 1], g[:j + 2], rcond=None)[0]
            if np.linalg.norm(H[:j + 2, :j + 1] @ y - g[:j + 2]) / bn <= 0.5 * tol or tot >= maxit:
                break
        x = x + V[:, :j + 1] @ y
    r = b - AP @ x
    return (x if P is None else P @ x), tot, np.linalg.norm(r) / bn <= tol
