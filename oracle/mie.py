"""Mie series for a homogeneous dielectric sphere (oracle side).

The paper validates the MTF against the Mie series (Sec. 5.2, citing the
absorption/scattering textbook of Bohren & Huffman).  This module restates
the textbook solution: Riccati-Bessel functions psi_n = rho j_n,
xi_n = rho h_n^(1) (time dependence exp(-i omega t)), coefficients

  a_n = [m psi_n(mx) psi_n'(x) - psi_n(x) psi_n'(mx)] / [m psi_n(mx) xi_n'(x) - xi_n(x) psi_n'(mx)]
  b_n = [psi_n(mx) psi_n'(x) - m psi_n(x) psi_n'(mx)] / [psi_n(mx) xi_n'(x) - m xi_n(x) psi_n'(mx)]

(mu_r = 1, m = sqrt(eps_r), x = k0 a), amplitude functions
S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n), S2 = sum ... (a_n tau_n + b_n pi_n),
and the far field of the incidence E = e1 exp(i k z):
E_sc ~ exp(i k r) / (-i k r) [cos(phi) S2 e_theta - sin(phi) S1 e_phi].
"""
from __future__ import annotations

import numpy as np


def _riccati_bessel(nmax, z):
    """psi_n(z), psi_n'(z) for n = 0..nmax by downward recurrence of j_n
    (Miller's algorithm normalised by j_0 = sin z / z)."""
    z = complex(z)
    nstart = nmax + 20 + int(abs(z))
    j = np.zeros(nstart + 2, dtype=np.complex128)
    j[nstart + 1] = 0.0
    j[nstart] = 1e-30
    for n in range(nstart, 0, -1):
        j[n - 1] = (2 * n + 1) / z * j[n] - j[n + 1]
    j *= (np.sin(z) / z) / j[0]
    psi = z * j[:nmax + 1]
    dpsi = np.empty_like(psi)
    dpsi[0] = np.cos(z)
    for n in range(1, nmax + 1):
        dpsi[n] = psi[n - 1] - n * psi[n] / z
    return psi, dpsi


def _riccati_hankel(nmax, x):
    """xi_n(x) = x h_n^(1)(x) and its derivative for real x > 0 (upward
    recurrence for y_n, stable)."""
    psi, dpsi = _riccati_bessel(nmax, x)
    y = np.zeros(nmax + 2)
    y[0] = -np.cos(x) / x
    y[1] = -np.cos(x) / x ** 2 - np.sin(x) / x
    for n in range(1, nmax):
        y[n + 1] = (2 * n + 1) / x * y[n] - y[n - 1]
    chi = x * y[:nmax + 1]
    dchi = np.empty_like(chi)
    dchi[0] = np.sin(x)  # d/dx (-cos x)
    for n in range(1, nmax + 1):
        dchi[n] = chi[n - 1] - n * chi[n] / x
    return psi + 1j * chi, dpsi + 1j * dchi


def mie_coefficients(k0, radius, eps_r, nmax=None):
    x = k0 * radius
    m = np.sqrt(complex(eps_r))
    if nmax is None:
        nmax = int(x + 4.05 * x ** (1 / 3) + 2) + 4
    px, dpx = _riccati_bessel(nmax, x)
    pmx, dpmx = _riccati_bessel(nmax, m * x)
    xx, dxx = _riccati_hankel(nmax, x)
    n = np.arange(1, nmax + 1)
    a = (m * pmx[n] * dpx[n] - px[n] * dpmx[n]) / (m * pmx[n] * dxx[n] - xx[n] * dpmx[n])
    b = (pmx[n] * dpx[n] - m * px[n] * dpmx[n]) / (pmx[n] * dxx[n] - m * xx[n] * dpmx[n])
    return a, b


def amplitude_functions(a, b, mu):
    """S1(mu), S2(mu), mu = cos(theta) (array)."""
    mu = np.asarray(mu, dtype=np.float64)
    nmax = len(a)
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    S1 = np.zeros(mu.shape, dtype=np.complex128)
    S2 = np.zeros(mu.shape, dtype=np.complex128)
    for n in range(1, nmax + 1):
        tau = n * mu * pi_cur - (n + 1) * pi_prev
        c = (2 * n + 1) / (n * (n + 1))
        S1 += c * (a[n - 1] * pi_cur + b[n - 1] * tau)
        S2 += c * (a[n - 1] * tau + b[n - 1] * pi_cur)
        pi_next = ((2 * n + 1) * mu * pi_cur - (n + 1) * pi_prev) / n
        pi_prev, pi_cur = pi_cur, pi_next
    return S1, S2


def mie_farfield(k0, radius, eps_r, d, p, obs):
    """Far field E_inf (n_obs, 3) of a sphere (centre 0) for E_inc = p exp(i k0 d.x),
    normalised as E_sc(x) ~ exp(i k0 |x|) / |x| E_inf(xhat).  p may be complex
    (linear in p; decomposed on a real basis orthogonal to d)."""
    d = np.asarray(d, dtype=np.float64) / np.linalg.norm(d)
    p = np.asarray(p, dtype=np.complex128)
    obs = np.atleast_2d(np.asarray(obs, dtype=np.float64))
    a, b = mie_coefficients(k0, radius, eps_r)
    ref = np.array([0.0, 0.0, 1.0]) if abs(d[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u1 = np.cross(ref, d)
    u1 /= np.linalg.norm(u1)
    u2 = np.cross(d, u1)
    out = np.zeros((len(obs), 3), dtype=np.complex128)
    mu = np.clip(obs @ d, -1.0, 1.0)
    S1, S2 = amplitude_functions(a, b, mu)
    for e1, coef in ((u1, p @ u1), (u2, p @ u2)):
        e2 = np.cross(d, e1)
        cx, cy = obs @ e1, obs @ e2
        phi = np.arctan2(cy, cx)
        st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
        # spherical unit vectors in the frame (e1, e2, d)
        eth = (mu * np.cos(phi))[:, None] * e1 + (mu * np.sin(phi))[:, None] * e2 - st[:, None] * d
        eph = -np.sin(phi)[:, None] * e1 + np.cos(phi)[:, None] * e2
        F = (1.0 / (-1j * k0)) * ((np.cos(phi) * S2)[:, None] * eth - (np.sin(phi) * S1)[:, None] * eph)
        out += coef * F
    return out
