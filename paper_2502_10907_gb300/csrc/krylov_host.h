// Host side of the batched GMRES: Hessenberg columns, complex Givens
// rotations, residual estimates and the small triangular solves, one
// Krylov space per right-hand side.  Used by the FP32-basis inner core.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace mtf {

struct HostArnoldi {
  using cd = std::complex<double>;
  int m = 0, nrhs = 0;
  std::vector<cd> H, g, sn;
  std::vector<double> cs, bnorm;
  std::vector<int> jc;
  HostArnoldi(int m_, int nrhs_) : m(m_), nrhs(nrhs_) {
    H.assign(size_t(m + 1) * m * nrhs, cd(0));
    g.assign(size_t(m + 1) * nrhs, cd(0));
    sn.assign(size_t(m) * nrhs, cd(0));
    cs.assign(size_t(m) * nrhs, 0.0);
    bnorm.assign(nrhs, 1.0);
    jc.assign(nrhs, 0);
  }
  // start of a cycle for rhs c with first basis vector r / ||r||; estimates
  // are relative to base (default ||r||)
  void start(int c, double rnorm, double base = -1.0) {
    jc[c] = 0;
    if (base < 0) base = rnorm;
    bnorm[c] = base > 0 ? base : 1.0;
    for (int q = 0; q <= m; ++q) g[size_t(c) * (m + 1) + q] = 0.0;
    g[size_t(c) * (m + 1)] = rnorm;
  }
  // Q (rows x k, column-major, ld = k + 1) and R (k x k upper triangular,
  // column-major, ld = ldr) of H = Q R for the first k columns of rhs c:
  // R is the rotated Hessenberg, Q = G_0^H ... G_{k-1}^H [I_k; 0]
  void qr(int c, int k, std::complex<double>* Q, std::complex<double>* R, int ldr) const {
    const cd* Hc = &H[size_t(c) * (m + 1) * m];
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q) R[size_t(p) * ldr + q] = q <= p ? Hc[size_t(p) * (m + 1) + q] : cd(0);
    const int ld = k + 1;
    for (int p = 0; p < k; ++p)
      for (int q = 0; q <= k; ++q) Q[size_t(p) * ld + q] = q == p ? cd(1) : cd(0);
    for (int j = k - 1; j >= 0; --j) {
      const double cj = cs[size_t(c) * m + j];
      const cd sj = sn[size_t(c) * m + j];
      for (int p = 0; p < k; ++p) {
        const cd a = Q[size_t(p) * ld + j], b = Q[size_t(p) * ld + j + 1];
        Q[size_t(p) * ld + j] = cj * a - sj * b;
        Q[size_t(p) * ld + j + 1] = std::conj(sj) * a + cj * b;
      }
    }
  }
  // column j of rhs c from h (interleaved complex, j+1 entries) and ||w||;
  // returns the relative residual estimate |g_{j+1}| / ||b||
  double add_column(int c, int j, const double* h, double hnorm) {
    cd* Hc = &H[size_t(c) * (m + 1) * m + size_t(j) * (m + 1)];
    for (int q = 0; q <= j; ++q) Hc[q] = cd(h[2 * q], h[2 * q + 1]);
    Hc[j + 1] = cd(hnorm, 0.0);
    for (int q = 0; q < j; ++q) {
      const double cq = cs[size_t(c) * m + q];
      const cd sq = sn[size_t(c) * m + q];
      const cd t = cq * Hc[q] + sq * Hc[q + 1];
      Hc[q + 1] = -std::conj(sq) * Hc[q] + cq * Hc[q + 1];
      Hc[q] = t;
    }
    const cd a = Hc[j], bb = Hc[j + 1];
    const double an = std::abs(a), bn = std::abs(bb), tt = std::hypot(an, bn);
    double cj;
    cd sj;
    if (tt == 0) {
      cj = 1.0;
      sj = 0.0;
    } else if (an == 0) {
      cj = 0.0;
      sj = std::conj(bb) / tt;
      Hc[j] = tt;
    } else {
      cj = an / tt;
      sj = (a / an) * std::conj(bb) / tt;
      Hc[j] = (a / an) * tt;
    }
    Hc[j + 1] = 0.0;
    cs[size_t(c) * m + j] = cj;
    sn[size_t(c) * m + j] = sj;
    cd* gc = &g[size_t(c) * (m + 1)];
    gc[j + 1] = -std::conj(sj) * gc[j];
    gc[j] = cj * gc[j];
    jc[c] = j + 1;
    return std::abs(gc[j + 1]) / bnorm[c];
  }
  // y = R^{-1} g of every rhs into yhost ((m+1) complex per rhs); returns max j
  int solve(std::vector<double>& yhost) const {
    std::fill(yhost.begin(), yhost.end(), 0.0);
    int jmax = 0;
    for (int c = 0; c < nrhs; ++c) {
      const int jj = jc[c];
      jmax = std::max(jmax, jj);
      const cd* Hc = &H[size_t(c) * (m + 1) * m];
      std::vector<cd> yy(jj);
      for (int q = jj - 1; q >= 0; --q) {
        cd acc = g[size_t(c) * (m + 1) + q];
        for (int p = q + 1; p < jj; ++p) acc -= Hc[size_t(p) * (m + 1) + q] * yy[p];
        yy[q] = acc / Hc[size_t(q) * (m + 1) + q];
      }
      for (int q = 0; q < jj; ++q) {
        yhost[2 * (size_t(c) * (m + 1) + q)] = yy[q].real();
        yhost[2 * (size_t(c) * (m + 1) + q) + 1] = yy[q].imag();
      }
    }
    return jmax;
  }
};

}  // namespace mtf
