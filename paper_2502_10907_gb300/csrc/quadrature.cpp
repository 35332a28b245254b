// Quadrature rules of the assembly, generated from their defining equations.
//
// The paper assembles with Bempp-cl defaults (Sec. 5.1) without stating the
// rules; the library uses
//  * regular (vertex-disjoint) pairs: tensor product of the fully symmetric
//    6-point degree-4 triangle rule, solved here from its moment equations;
//  * singular pairs: the Sauter-Schwab transformations (Sauter & Schwab,
//    Boundary Element Methods, Sec. 5.2) of K x K, K = {0 <= x2 <= x1 <= 1},
//    onto [0,1]^4 with an n-point Gauss-Legendre rule per coordinate.
#include <cmath>
#include <mutex>

#include "common.h"

namespace mtf {

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton on P_n with the three-term recurrence; nodes ascending on [0, 1].
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    // roots come out descending in z, so x = (1 - z) / 2 is ascending
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

static void tri6_solve(TriRule& r) {
  // unknowns (a, b, wa, wb); residual of the invariant moments 1, e2, e3, e2^2
  const double target[4] = {0.5, 1.0 / 8.0, 1.0 / 120.0, 1.0 / 30.0};
  auto inv = [](double a, double* f) {
    double e2 = 2 * a - 3 * a * a, e3 = a * a * (1 - 2 * a);
    f[0] = 1.0; f[1] = e2; f[2] = e3; f[3] = e2 * e2;
  };
  auto F = [&](const double* z, double* out) {
    double fa[4], fb[4];
    inv(z[0], fa);
    inv(z[1], fb);
    for (int q = 0; q < 4; ++q) out[q] = 3 * z[2] * fa[q] + 3 * z[3] * fb[q] - target[q];
  };
  double z[4] = {0.44, 0.09, 0.11, 0.055};
  for (int it = 0; it < 60; ++it) {
    double f[4], J[4][4];
    F(z, f);
    for (int c = 0; c < 4; ++c) {
      double zp[4], zm[4], fp[4], fm[4];
      for (int q = 0; q < 4; ++q) zp[q] = zm[q] = z[q];
      zp[c] += 1e-7;
      zm[c] -= 1e-7;
      F(zp, fp);
      F(zm, fm);
      for (int q = 0; q < 4; ++q) J[q][c] = (fp[q] - fm[q]) / 2e-7;
    }
    // Gaussian elimination with partial pivoting on J dz = f
    double A[4][5];
    for (int q = 0; q < 4; ++q) {
      for (int c = 0; c < 4; ++c) A[q][c] = J[q][c];
      A[q][4] = f[q];
    }
    for (int c = 0; c < 4; ++c) {
      int piv = c;
      for (int q = c + 1; q < 4; ++q)
        if (std::fabs(A[q][c]) > std::fabs(A[piv][c])) piv = q;
      for (int cc = 0; cc < 5; ++cc) std::swap(A[c][cc], A[piv][cc]);
      for (int q = c + 1; q < 4; ++q) {
        double m = A[q][c] / A[c][c];
        for (int cc = c; cc < 5; ++cc) A[q][cc] -= m * A[c][cc];
      }
    }
    double dz[4];
    for (int c = 3; c >= 0; --c) {
      double s = A[c][4];
      for (int cc = c + 1; cc < 4; ++cc) s -= A[c][cc] * dz[cc];
      dz[c] = s / A[c][c];
    }
    double mx = 0;
    for (int q = 0; q < 4; ++q) {
      z[q] -= dz[q];
      mx = std::fmax(mx, std::fabs(dz[q]));
    }
    if (mx < 1e-15) break;
  }
  int p = 0;
  const double orb[2] = {z[0], z[1]}, ow[2] = {z[2], z[3]};
  for (int o = 0; o < 2; ++o) {
    double c = orb[o];
    const double lam[3][3] = {{1 - 2 * c, c, c}, {c, 1 - 2 * c, c}, {c, c, 1 - 2 * c}};
    for (int q = 0; q < 3; ++q) {
      r.s[p] = lam[q][1];
      r.t[p] = lam[q][2];
      r.w[p] = ow[o];
      ++p;
    }
  }
}

const TriRule& triangle_rule6() {
  static TriRule rule;
  static std::once_flag once;
  std::call_once(once, [] { tri6_solve(rule); });
  return rule;
}

void sauter_schwab_rule(int kind, int n, std::vector<double>& pts) {
  std::vector<double> g, gw;
  gauss_legendre01(n, g, gw);
  const int nreg = kind == 0 ? 6 : (kind == 1 ? 5 : 2);
  pts.clear();
  pts.reserve(size_t(nreg) * n * n * n * n * 5);
  for (int reg = 0; reg < nreg; ++reg) {
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c)
          for (int d = 0; d < n; ++d) {
            const double xi = g[a], e1 = g[b], e2 = g[c], e3 = g[d];
            const double W = gw[a] * gw[b] * gw[c] * gw[d];
            double x1 = 0, x2 = 0, y1 = 0, y2 = 0, J = 0;
            if (kind == 0) {  // coincident: Jacobian xi^3 eta1^2 eta2
              J = xi * xi * xi * e1 * e1 * e2;
              switch (reg) {
                case 0: x1 = xi; x2 = xi * (1 - e1 + e1 * e2); y1 = xi * (1 - e1 * e2 * e3); y2 = xi * (1 - e1); break;
                case 1: y1 = xi; y2 = xi * (1 - e1 + e1 * e2); x1 = xi * (1 - e1 * e2 * e3); x2 = xi * (1 - e1); break;
                case 2: x1 = xi; x2 = xi * e1 * (1 - e2 + e2 * e3); y1 = xi * (1 - e1 * e2); y2 = xi * e1 * (1 - e2); break;
                case 3: y1 = xi; y2 = xi * e1 * (1 - e2 + e2 * e3); x1 = xi * (1 - e1 * e2); x2 = xi * e1 * (1 - e2); break;
                case 4: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * e1 * (1 - e2 * e3); y1 = xi; y2 = xi * e1 * (1 - e2); break;
                default: y1 = xi * (1 - e1 * e2 * e3); y2 = xi * e1 * (1 - e2 * e3); x1 = xi; x2 = xi * e1 * (1 - e2); break;
              }
            } else if (kind == 1) {  // common edge P0-P1 (x2 = 0 in both)
              J = reg == 0 ? xi * xi * xi * e1 * e1 : xi * xi * xi * e1 * e1 * e2;
              switch (reg) {
                case 0: x1 = xi; x2 = xi * e1 * e3; y1 = xi * (1 - e1 * e2); y2 = xi * e1 * (1 - e2); break;
                case 1: x1 = xi; x2 = xi * e1; y1 = xi * (1 - e1 * e2 * e3); y2 = xi * e1 * e2 * (1 - e3); break;
                case 2: x1 = xi * (1 - e1 * e2); x2 = xi * e1 * (1 - e2); y1 = xi; y2 = xi * e1 * e2 * e3; break;
                case 3: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * e1 * e2 * (1 - e3); y1 = xi; y2 = xi * e1; break;
                default: x1 = xi * (1 - e1 * e2 * e3); x2 = xi * e1 * (1 - e2 * e3); y1 = xi; y2 = xi * e1 * e2; break;
              }
            } else {  // common vertex P0 (origin of both)
              J = xi * xi * xi * e2;
              if (reg == 0) { x1 = xi; x2 = xi * e1; y1 = xi * e2; y2 = xi * e2 * e3; }
              else { x1 = xi * e2; x2 = xi * e2 * e3; y1 = xi; y2 = xi * e1; }
            }
            pts.push_back(x1);
            pts.push_back(x2);
            pts.push_back(y1);
            pts.push_back(y2);
            pts.push_back(W * J);
          }
  }
}

}  // namespace mtf
