// Host checks of the block-GMRES helpers (block_krylov.h):
//  1. deflating_cholesky on a block with a dependent column: the kept
//     columns of V = W T are orthonormal, W = V R, the dependent column is
//     deflated;
//  2. BlockLSQ on random block upper-Hessenberg matrices, blocks of 4 and of
//     32 columns (with the zero rows
//     and columns a deflated direction gives): the coefficients Y solve the
//     least-squares problem min ||E_1 S_0 - Hbar Y|| (compared with the
//     normal equations solved densely) and the residual estimates equal the
//     true residual norms;
//  3. the worker pool gives the single-thread results (below).
#include <cstdio>
#include <random>
#include "block_krylov.h"
using cd = std::complex<double>;

static double check_cholesky() {
  const int n = 40, s = 5;
  std::mt19937 rng(7);
  std::normal_distribution<double> N(0, 1);
  std::vector<cd> W(size_t(n) * s);
  for (auto& v : W) v = cd(N(rng), N(rng));
  for (int i = 0; i < n; ++i) W[size_t(3) * n + i] = 2.0 * W[size_t(1) * n + i] - cd(0, 1) * W[i];  // dependent
  std::vector<cd> G(size_t(s) * s), R(size_t(s) * s), T(size_t(s) * s);
  std::vector<double> ref(s);
  for (int a = 0; a < s; ++a)
    for (int b = 0; b < s; ++b) {
      cd acc = 0;
      for (int i = 0; i < n; ++i) acc += std::conj(W[size_t(a) * n + i]) * W[size_t(b) * n + i];
      G[size_t(b) * s + a] = acc;
    }
  for (int a = 0; a < s; ++a) ref[a] = G[size_t(a) * s + a].real();
  std::vector<int> kept;
  const int nk = mtf::deflating_cholesky(s, G.data(), ref.data(), 1e-6, R.data(), T.data(), kept);
  std::vector<cd> V(size_t(n) * s, 0.0);
  for (int q = 0; q < s; ++q)
    for (int c = 0; c < s; ++c)
      for (int i = 0; i < n; ++i) V[size_t(q) * n + i] += W[size_t(c) * n + i] * T[size_t(q) * s + c];
  double orth = 0, rec = 0, nw = 0;
  for (int a = 0; a < s; ++a)
    for (int b = 0; b < s; ++b) {
      cd acc = 0;
      for (int i = 0; i < n; ++i) acc += std::conj(V[size_t(a) * n + i]) * V[size_t(b) * n + i];
      const double want = (a == b && kept[a]) ? 1.0 : 0.0;
      orth = std::max(orth, std::abs(acc - want));
    }
  for (int c = 0; c < s; ++c)
    for (int i = 0; i < n; ++i) {
      cd acc = 0;
      for (int q = 0; q < s; ++q) acc += V[size_t(q) * n + i] * R[size_t(c) * s + q];
      rec += std::norm(acc - W[size_t(c) * n + i]);
      nw += std::norm(W[size_t(c) * n + i]);
    }
  std::printf("cholesky: kept %d of %d (deflated col 3: %d)  ||V^H V - I||max = %.2e  ||VR - W||/||W|| = %.2e\n", nk, s,
              int(!kept[3]), orth, std::sqrt(rec / nw));
  return (nk == s - 1 && !kept[3] && orth < 1e-10 && std::sqrt(rec / nw) < 1e-10) ? 0.0 : 1.0;
}

static double check_lsq(int s, int kb) {
  const int m = kb + 3;
  std::mt19937 rng(11);
  std::normal_distribution<double> N(0, 1);
  const int rows = (kb + 1) * s, cols = kb * s;
  std::vector<cd> H(size_t(rows) * cols, 0.0), S0(size_t(s) * s, 0.0);
  for (int c = 0; c < s; ++c)
    for (int i = 0; i <= c; ++i) S0[size_t(c) * s + i] = cd(N(rng), N(rng));
  mtf::BlockLSQ L;
  std::vector<double> bn(s, 1.0);
  L.init(s, m, S0.data(), bn.data());
  std::vector<double> est(s);
  for (int j = 0; j < kb; ++j) {
    std::vector<cd> h(size_t(j + 1) * s * s), R(size_t(s) * s, 0.0);
    for (auto& v : h) v = cd(N(rng), N(rng));
    for (int c = 0; c < s; ++c)
      for (int i = 0; i <= c; ++i) R[size_t(c) * s + i] = cd(N(rng), N(rng));
    // direction 2 deflated from V_3 on, as block Arnoldi produces it: row 2
    // of R_3 is zero; from block 3 on, Z column 2 is zero (zero column of h
    // and R, zero row 2 of R), and V_q column 2 (q >= 3) is zero, so rows
    // 3 s + 2, 4 s + 2, ... of h vanish
    if (j >= 2)
      for (int c = 0; c < s; ++c) R[size_t(c) * s + 2] = 0.0;
    if (j >= 3) {
      for (int i = 0; i < (j + 1) * s; ++i) h[size_t(2) * (j + 1) * s + i] = 0.0;
      for (int i = 0; i < s; ++i) R[size_t(2) * s + i] = 0.0;
      for (int c = 0; c < s; ++c)
        for (int q = 3; q <= j; ++q) h[size_t(c) * (j + 1) * s + q * s + 2] = 0.0;
    }
    for (int c = 0; c < s; ++c) {
      for (int i = 0; i < (j + 1) * s; ++i) H[size_t(j * s + c) * rows + i] = h[size_t(c) * (j + 1) * s + i];
      for (int i = 0; i < s; ++i) H[size_t(j * s + c) * rows + (j + 1) * s + i] = R[size_t(c) * s + i];
    }
    L.add_block(h.data(), j + 1, R.data(), est.data());
  }
  std::vector<cd> Y;
  L.solve(Y);
  // true residuals and the normal equations (H^H H) Y = H^H E S0, zero column excluded
  double worst_est = 0, worst_ne = 0;
  for (int c = 0; c < s; ++c) {
    std::vector<cd> r(rows, 0.0);
    for (int i = 0; i < s; ++i) r[i] = S0[size_t(c) * s + i];
    for (int p = 0; p < cols; ++p)
      for (int i = 0; i < rows; ++i) r[i] -= H[size_t(p) * rows + i] * Y[size_t(c) * cols + p];
    double rn = 0;
    for (auto& v : r) rn += std::norm(v);
    worst_est = std::max(worst_est, std::abs(std::sqrt(rn) - est[c]) / std::max(1e-300, est[c]));
    for (int p = 0; p < cols; ++p) {  // gradient H^H r must vanish
      cd acc = 0;
      for (int i = 0; i < rows; ++i) acc += std::conj(H[size_t(p) * rows + i]) * r[i];
      worst_ne = std::max(worst_ne, std::abs(acc));
    }
  }
  std::printf("lsq (s = %d, %d blocks): max |est - ||r||| / est = %.2e   max |H^H r| = %.2e\n", s, kb, worst_est,
              worst_ne);
  return (worst_est < 1e-10 && worst_ne < 1e-10) ? 0.0 : 1.0;
}

// 3. the same updates on the host worker pool: 40 column blocks of 16
//    columns (past the size at which BlockLSQ hands its columns to the pool;
//    the least-squares solve too), once on 1 thread and once on 4, give
//    bit-identical estimates and coefficients (every column follows the same
//    arithmetic on whichever thread runs it)
static double check_pool() {
  const int s = 16, kb = 40, m = 44;
  std::vector<std::vector<cd>> hs, Rs;
  std::mt19937 rng(13);
  std::normal_distribution<double> N(0, 1);
  for (int j = 0; j < kb; ++j) {
    std::vector<cd> h(size_t(j + 1) * s * s), R(size_t(s) * s, 0.0);
    for (auto& v : h) v = cd(N(rng), N(rng));
    for (int c = 0; c < s; ++c)
      for (int i = 0; i <= c; ++i) R[size_t(c) * s + i] = cd(N(rng), N(rng)) * (i == c ? 4.0 : 1.0);
    hs.push_back(h);
    Rs.push_back(R);
  }
  std::vector<cd> S0(size_t(s) * s, 0.0);
  for (int c = 0; c < s; ++c) S0[size_t(c) * s + c] = 1.0 + c;
  std::vector<double> bn(s, 1.0);
  std::vector<double> est[2];
  std::vector<cd> Y[2];
  int rounds = 0;
  for (int v = 0; v < 2; ++v) {
    mtf::BlockLSQ L;
    L.init(s, m, S0.data(), bn.data());
    L.threads = v == 0 ? 1 : 4;
    est[v].assign(s, 0.0);
    for (int r = 0; r < 3; ++r) {  // the pool serves several solves in a row
      L.init(s, m, S0.data(), bn.data());
      L.threads = v == 0 ? 1 : 4;
      for (int j = 0; j < kb; ++j) L.add_block(hs[j].data(), j + 1, Rs[j].data(), est[v].data());
      L.solve(Y[v]);
      rounds += v;
    }
  }
  bool same = Y[0].size() == Y[1].size();
  for (size_t i = 0; same && i < Y[0].size(); ++i) same = Y[0][i] == Y[1][i];
  for (int c = 0; same && c < s; ++c) same = est[0][c] == est[1][c];
  std::printf("pool: %d pooled solves, results %s\n", rounds, same ? "identical" : "DIFFER");
  return same ? 0.0 : 1.0;
}

int main() {
  // s = 4: reflectors of earlier blocks applied to column pairs; s = 32:
  // in groups of 4 columns
  const double f = check_cholesky() + check_lsq(4, 7) + check_lsq(32, 6) + check_pool();
  return f == 0.0 ? 0 : 1;
}
