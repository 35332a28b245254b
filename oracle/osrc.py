"""Block-OSRC preconditioner (oracle side), Sec. 4.4 of the paper.

The paper defines the block preconditioner
    A~_i = [[0, rho_i^-1 T~], [-rho_i T~, 0]]          (Eq. 19)
with T~ = Pi~^{-1}_{k, eps, N_p} an OSRC approximation of the EtM map
EtM = -T^{-1}(I/2 + K), built from a Pade approximation (order N_p, damped
wavenumber k_eps = k + i eps) of a square-root surface operator, and leaves
its discretisation to the cited OSRC work.  Reading taken here (stated in
the design notes; the CUDA library implements the same operator):

* Principal symbols of the Galerkin EFIO on a flat patch (outgoing branch
  q = sqrt(|xi|^2 - k^2)): on irrotational currents (grad phi) the EFIO acts
  as i q / (2k), on solenoidal currents (n x grad phi) as -i k / (2q).  With
  k_eps = k + i eps and Z = -|xi|^2 / k_eps^2 their inverses are
      irrotational:  2k / (k_eps sqrt(1 + Z)),
      solenoidal:    (2 k_eps / k) sqrt(1 + Z),
  the two factors of the OSRC magnetic-to-electric operator
  (1 + X/k_eps^2)^{-1/2} (1 - curl curl / k_eps^2), X the surface Hodge
  Laplacian; both tend to 2 as |xi| -> 0.
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
* Discretisation on RWG_i (closed, connected Gamma_i of genus g): the RWG
  space splits G-orthogonally into the irrotational part (generalised
  eigenpairs D v = lambda G v with lambda > 0, D the div-div and G the mass
  matrix; |xi|^2 = lambda), the loop part, the RWG images u = L phi of nodal
  P1 functions (u = n x grad phi exactly, L[e, lo] = 1/l_e,
  L[e, hi] = -1/l_e), whose eigenpairs S phi = mu M phi (P1 stiffness S,
  mass M; |xi|^2 = mu) give G-orthonormal loop modes L phi / sqrt(mu)
  (L^T G L = S), and, when g > 0, the 2 g discrete harmonic fields: the part
  of the kernel of D that is G-orthogonal to the loops (by Euler's formula
  its dimension is N - (T - 1) - (V - 1) = 2 g).  Harmonic fields are both
  divergence- and curl-free, so their symbol is the loop symbol at
  |xi|^2 = 0; T~ does not depend on the basis chosen for them.  With W the
  G-orthonormal basis of all parts and f the matching symbols,
      T~ = W diag(f) W^T,
  which maps tested vectors to coefficients (W W^T = G^{-1}); the Pade
  approximant is applied exactly on every mode instead of through auxiliary
  sparse solves.
* Type 2 (Sec. 5.4 uses it and only cites its source, for a twofold saving in
  memory and solver time at similar iteration counts; no definition is
  printed).  Reading taken here: a compressed T~ whose modal symbols keep
  their modulus and take the phase of the principal symbols of the EtM map
  (the |xi| -> infinity limits -2ik/|xi| on irrotational and 2i|xi|/k on
  solenoidal currents, i.e. -pi/2 and +pi/2):
      f2 = -i |f| on irrotational modes,  f2 = +i |f| on loop and harmonic
      modes,   T~2 = W diag(f2) W^T = i R,  R = W diag(Im f2) W^T real.
  R is real symmetric, so T~2 needs half the storage of T~ and its apply to
  a complex vector is two real products.  For the damped symbols used here
  the irrotational symbols have Im f < 0 and the solenoidal ones Im f > 0,
  so f2 = i sign(Im f) |f|: Type 2 rounds every symbol's phase to the
  nearest of +-pi/2.  It changes iteration counts only, never the solution.
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


def p1_matrices(sk: Skeleton, i: int):
    """Vertices of Gamma_i and the P1 Laplace-Beltrami stiffness S and mass M."""
    tris = sk.tris[i]
    F = sk.F[tris]
    verts = np.unique(F)
    pos = {v: q for q, v in enumerate(verts)}
    nv = len(verts)
    S = np.zeros((nv, nv))
    M = np.zeros((nv, nv))
    for t in range(len(tris)):
        f = F[t]
        P = sk.V[f]
        A = sk.area[tris[t]]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        g = [np.cross(n, P[(a + 2) % 3] - P[(a + 1) % 3]) / (n @ n) for a in range(3)]
        for a in range(3):
            for b in range(3):
                S[pos[f[a]], pos[f[b]]] += A * (g[a] @ g[b])
                M[pos[f[a]], pos[f[b]]] += A * (2.0 if a == b else 1.0) / 12.0
    return verts, pos, S, M


def loop_map(sk: Skeleton, i: int, pos):
    """L[e, v]: RWG coefficients of n_i x grad(phi_v), L[e, lo] = 1/l, L[e, hi] = -1/l."""
    E = sk.edges[i]
    L = np.zeros((len(E), len(pos)))
    le = np.linalg.norm(sk.V[E[:, 1]] - sk.V[E[:, 0]], axis=1)
    for e, (lo, hi) in enumerate(E):
        L[e, pos[lo]] = 1.0 / le[e]
        L[e, pos[hi]] = -1.0 / le[e]
    return L


class BlockOSRC:
    """Block-OSRC preconditioner of an MTF system (Eq. 19)."""

    def __init__(self, sk: Skeleton, k, rho, Np=4, theta=np.pi / 2, eps_scale=0.39, osrc_type=1):
        if osrc_type not in (1, 2):
            raise ValueError("block-OSRC type must be 1 or 2")
        self.sk = sk
        self.rho = np.asarray(rho)
        self.osrc_type = osrc_type
        self.Ttil = []
        self.nh, self.W, self.f, self.n_irr = [], [], [], []
        for i in range(sk.n_domains):
            G = mass_matrix(sk, i)
            D = divdiv_matrix(sk, i)
            lam, V = scipy.linalg.eigh(D, G)
            nirr = len(sk.tris[i]) - 1                 # rank of div on RWG_i
            verts, pos, S, M = p1_matrices(sk, i)
            mu, Phi = scipy.linalg.eigh(S, M)
            nh = sk.N[i] - nirr - (len(verts) - 1)      # 2 g harmonic fields
            if nh < 0 or nh % 2:
                raise ValueError("block-OSRC needs connected subdomain boundaries")
            U = loop_map(sk, i, pos) @ Phi[:, 1:] / np.sqrt(mu[1:])[None, :]
            if nh:
                K = V[:, :sk.N[i] - nirr]                # kernel of D (G-orthonormal)
                R = K - U @ (U.T @ G @ K)                # its part G-orthogonal to the loops
                s2, Q = scipy.linalg.eigh(R.T @ G @ R)   # nh eigenvalues 1, the rest 0
                H = R @ Q[:, -nh:] / np.sqrt(s2[-nh:])[None, :]
                U = np.concatenate([U, H], axis=1)
                mu = np.concatenate([mu, np.zeros(nh)])
            area = float(np.sum(sk.area[sk.tris[i]]))
            keps = k[i] + 1j * damping(k[i], area, eps_scale)
            f_irr = 2 * k[i] / (keps * pade_sqrt(-lam[-nirr:] / keps ** 2, Np, theta))
            f_sol = (2 * keps / k[i]) * pade_sqrt(-mu[1:] / keps ** 2, Np, theta)
            W = np.concatenate([V[:, -nirr:], U], axis=1)
            f = np.concatenate([f_irr, f_sol])
            if osrc_type == 2:
                # Type 2: modulus kept, phase of the principal symbol
                # (-pi/2 irrotational, +pi/2 loops and harmonic fields)
                sigma = np.concatenate([-np.ones(nirr), np.ones(len(f_sol))])
                f = 1j * sigma * np.abs(f)
            self.nh.append(nh)
            self.n_irr.append(nirr)
            self.W.append(W)
            self.f.append(f)
            self.Ttil.append((W * f[None, :]) @ W.T)

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
