// Host checks of the tensor-core matvec plan and formulation (tc_plan.h):
//  1. plan_tc: every (block, row tile, chunk) lies in exactly one unit, the
//     units of (block, row tile) are consecutive from unit_base, the schedule
//     is a permutation of the units and its busiest CTA carries at most the
//     average plus one longest unit;
//  2. the formulation: T and K of a ragged block (N = 45, not a multiple of
//     the tile sizes) packed into the tiled FP16 hi / lo layout after
//     power-of-two scaling, the inputs packed into chunks in the two real
//     column forms, the products emulated as the tensor cores form them
//     (FP16 operands, hi*hi + hi*lo + lo*hi per chunk) and unscaled give
//     T u and K u to about 2^-22 of the exact complex products;
//  4. the block-OSRC formation plan (plan_tt): the formed units with the
//     in-place / mirror rule write every entry of every T~_i exactly once,
//     tile and chunk indices stay inside the allocations, and the formation
//     emulated in that layout (W and f^(t) W scaled, split into FP16 hi + lo,
//     three products, FP32 sums) gives W diag(f) W^T to about 2^-21;
//  3. the two tiled basis copies of the tensor-core Gram-Schmidt projections:
//     every (vector, entry, part) of the basis sizes used maps inside the
//     allocation (the stores write 8 halves from a multiple-of-4 entry), and
//     on a small basis the map is one to one.
#include <cmath>
#include <complex>
#include <cstdio>
#include <random>
#include "tc_plan.h"
using cd = std::complex<double>;

static int check_plan(const std::vector<int>& Ns, int ncta) {
  mtf::TcPlan p;
  const std::string why = mtf::plan_tc(Ns, ncta, p);
  if (!why.empty()) return std::printf("plan: %s\n", why.c_str()), 1;
  // coverage
  std::vector<int> seen(size_t(p.n_tiles), 0);
  int64_t longest = 0;
  for (size_t u = 0; u < p.units.size(); ++u) {
    const auto& U = p.units[u];
    const auto& b = p.blocks[size_t(U.blk)];
    longest = std::max<int64_t>(longest, U.kc1 - U.kc0);
    const int q = int(u) - b.unit_base - U.mt * b.pieces;
    if (q < 0 || q >= b.pieces || U.kc0 != q * b.piece_len) return std::printf("plan: unit order\n"), 1;
    for (int kc = U.kc0; kc < U.kc1; ++kc) ++seen[size_t(b.tile_base + int64_t(U.mt) * b.n_kc + kc)];
  }
  for (int v : seen)
    if (v != 1) return std::printf("plan: coverage\n"), 1;
  std::vector<int> cnt(p.units.size(), 0);
  for (int u : p.sched) ++cnt[size_t(u)];
  for (int v : cnt)
    if (v != 1) return std::printf("plan: schedule\n"), 1;
  const double avg = double(p.total_load) / ncta;
  std::printf("plan: %zu blocks, %zu units, max load %lld chunks (avg %.1f, longest unit %lld)\n", Ns.size(),
              p.units.size(), (long long)p.max_load, avg, (long long)longest);
  return p.max_load <= avg + longest ? 0 : 1;
}

static float f16(float v) { return float(_Float16(v)); }

static int check_formulation() {
  const int N = 45, nc = 3;
  std::mt19937 rng(5);
  std::normal_distribution<double> G(0, 1);
  std::vector<std::complex<float>> T(size_t(N) * N), K(size_t(N) * N), u(size_t(2 * N) * nc);
  for (auto& v : T) v = {float(G(rng) * 3e-3), float(G(rng) * 3e-3)};
  for (auto& v : K) v = {float(G(rng) * 1e-2), float(G(rng) * 1e-2)};
  for (auto& v : u) v = {float(G(rng)), float(G(rng))};
  mtf::TcPlan p;
  mtf::plan_tc({N}, 4, p);
  const auto& b = p.blocks[0];
  const int nb = mtf::tc_nb(nc);
  // scales (largest |re|, |im| mapped below 2^14)
  auto scale = [](double amax) { int ex; std::frexp(amax, &ex); return std::ldexp(1.0, 14 - ex); };
  double am = 0;
  for (int t = 0; t < N * N; ++t)
    am = std::max({am, double(std::fabs(T[t].real())), double(std::fabs(T[t].imag())), double(std::fabs(K[t].real())),
                   double(std::fabs(K[t].imag()))});
  const float sA = float(scale(am));
  std::vector<float> sB(nc);
  for (int c = 0; c < nc; ++c) {
    double m = 0;
    for (int k = 0; k < 2 * N; ++k) m = std::max({m, double(std::fabs(u[size_t(c) * 2 * N + k].real())),
                                                  double(std::fabs(u[size_t(c) * 2 * N + k].imag()))});
    sB[c] = float(scale(m));
  }
  std::vector<float> A(size_t(p.n_tiles * mtf::kTcTileHalves), 0.f), B(size_t(p.n_chunks) * 2 * nb * 64, 0.f);
  for (int mt = 0; mt < b.n_mt; ++mt)
    for (int kc = 0; kc < b.n_kc; ++kc)
      for (int row = 0; row < mtf::kTcRows; ++row)
        for (int q = 0; q < mtf::kTcCols; ++q) {
          const int r = mt * mtf::kTcRows + row, n = kc * mtf::kTcCols + q;
          if (r >= N || n >= N) continue;
          const int64_t tile = b.tile_base + int64_t(mt) * b.n_kc + kc;
          const float vals[4] = {T[size_t(r) * N + n].real() * sA, T[size_t(r) * N + n].imag() * sA,
                                 K[size_t(r) * N + n].real() * sA, K[size_t(r) * N + n].imag() * sA};
          for (int op = 0; op < 2; ++op)
            for (int ri = 0; ri < 2; ++ri) {
              const float v = vals[2 * op + ri], hi = f16(v), lo = f16(v - hi);
              A[size_t(mtf::tc_a_index(tile, 2 * op, row, 2 * q + ri))] = hi;
              A[size_t(mtf::tc_a_index(tile, 2 * op + 1, row, 2 * q + ri))] = lo;
            }
        }
  for (int kc = 0; kc < b.n_kc; ++kc)
    for (int col = 0; col < 4 * nc; ++col)
      for (int q = 0; q < mtf::kTcCols; ++q) {
        const int n = kc * mtf::kTcCols + q;
        if (n >= N) continue;
        const int c = col >> 2, slot = (col >> 1) & 1, form = col & 1;
        const std::complex<float> v = u[size_t(c) * 2 * N + size_t(slot) * N + n];
        const float pair[2] = {form == 0 ? v.real() : v.imag(), form == 0 ? -v.imag() : v.real()};
        for (int t = 0; t < 2; ++t) {
          const float x = pair[t] * sB[c], hi = f16(x), lo = f16(x - hi);
          B[size_t(mtf::tc_b_index(b.chunk_base + kc, 0, col, 2 * q + t, nb))] = hi;
          B[size_t(mtf::tc_b_index(b.chunk_base + kc, 1, col, 2 * q + t, nb))] = lo;
        }
      }
  // emulated products: D_op[row][col] += sum_e Ahi Bhi + Ahi Blo + Alo Bhi (FP32 sums)
  double err = 0, ref = 0;
  for (int mt = 0; mt < b.n_mt; ++mt)
    for (int row = 0; row < mtf::kTcRows; ++row) {
      const int r = mt * mtf::kTcRows + row;
      if (r >= N) continue;
      for (int op = 0; op < 2; ++op)
        for (int col = 0; col < 4 * nc; ++col) {
          float acc = 0.f;
          for (int kc = 0; kc < b.n_kc; ++kc) {
            const int64_t tile = b.tile_base + int64_t(mt) * b.n_kc + kc, ch = b.chunk_base + kc;
            for (int e = 0; e < 64; ++e) {
              const float ah = A[size_t(mtf::tc_a_index(tile, 2 * op, row, e))];
              const float al = A[size_t(mtf::tc_a_index(tile, 2 * op + 1, row, e))];
              const float bh = B[size_t(mtf::tc_b_index(ch, 0, col, e, nb))];
              const float bl = B[size_t(mtf::tc_b_index(ch, 1, col, e, nb))];
              acc += ah * bh + ah * bl + al * bh;
            }
          }
          const int c = col >> 2, slot = (col >> 1) & 1, form = col & 1;
          cd exact = 0;
          for (int n = 0; n < N; ++n) {
            const auto& M = op == 0 ? T : K;
            exact += cd(M[size_t(r) * N + n]) * cd(u[size_t(c) * 2 * N + size_t(slot) * N + n]);
          }
          const double want = form == 0 ? exact.real() : exact.imag();
          const double got = double(acc) / (double(sA) * sB[c]);
          err += (got - want) * (got - want);
          ref += want * want;
        }
    }
  const double rel = std::sqrt(err / ref);
  std::printf("formulation: ||emulated - exact|| / ||exact|| = %.2e\n", rel);
  return rel < 1e-6 ? 0 : 1;
}

static int check_basis_layout() {
  struct Case { int64_t ldn, nvec; };
  const Case cases[] = {{2880, 501 * 16}, {72000, 601 * 16}, {13120, 501 * 2}, {35008, 201 * 64}, {64, 3}};
  for (const Case& c : cases) {
    const int64_t nkc = c.ldn / mtf::kTcCols, nbc = (c.nvec + 31) / 32;
    const int64_t nd = mtf::tca_dots_halves(c.nvec, c.ldn), nu = mtf::tca_upd_halves(c.nvec, c.ldn);
    const int64_t qs[] = {0, 1, 31, 32, 127, 128, c.nvec - 2, c.nvec - 1};
    for (int64_t qq : qs) {
      if (qq < 0 || qq >= c.nvec) continue;
      for (int64_t k = 0; k < c.ldn; ++k)
        for (int part = 0; part < 2; ++part) {
          const int64_t d = mtf::tca_dots_half(qq, k & ~int64_t(3), nkc, part) + 7;
          const int64_t u = mtf::tca_upd_half(qq, k, nbc, part) + 1;
          if (d >= nd || u >= nu) {
            std::printf("basis layout: out of range (ldn %lld nvec %lld qq %lld k %lld)\n", (long long)c.ldn,
                        (long long)c.nvec, (long long)qq, (long long)k);
            return 1;
          }
        }
    }
  }
  // one to one on a small basis
  const int64_t ldn = 128, nvec = 64, nkc = ldn / mtf::kTcCols, nbc = (nvec + 31) / 32;
  std::vector<int> hd(size_t(mtf::tca_dots_halves(nvec, ldn)), 0), hu(size_t(mtf::tca_upd_halves(nvec, ldn)), 0);
  for (int64_t qq = 0; qq < nvec; ++qq)
    for (int64_t k = 0; k < ldn; ++k)
      for (int part = 0; part < 2; ++part)
        for (int ri = 0; ri < 2; ++ri) {
          ++hd[size_t(mtf::tca_dots_half(qq, k, nkc, part) + ri)];
          ++hu[size_t(mtf::tca_upd_half(qq, k, nbc, part) + ri)];
        }
  for (int v : hd)
    if (v > 1) return std::printf("basis layout: dots copy not one to one\n"), 1;
  for (int v : hu)
    if (v > 1) return std::printf("basis layout: update copy not one to one\n"), 1;
  std::printf("basis layout: in range for all cases, one to one on the small basis\n");
  return 0;
}

static float p2scale(double a) {
  if (!(a > 0)) return 1.f;
  int ex;
  std::frexp(a, &ex);
  return std::ldexp(1.f, 14 - ex);
}

// plan_tt coverage and index bounds; with emulate, the formation itself
static int check_tt(const std::vector<int>& Ns, bool emulate) {
  mtf::TtPlan p;
  const std::string why = mtf::plan_tt(Ns, p);
  if (!why.empty()) return std::printf("tt: %s\n", why.c_str()), 1;
  std::mt19937 rng(11);
  std::normal_distribution<double> G(0, 1);
  const int64_t na = p.n_a * 2 * mtf::kTcRows * 64, nb = p.n_b * 2 * 128 * 64;
  std::vector<float> A, B;
  std::vector<std::vector<double>> W(Ns.size());
  std::vector<std::vector<cd>> F(Ns.size());
  std::vector<float> inv(Ns.size());
  if (emulate) {
    A.assign(size_t(na), 0.f);
    B.assign(size_t(nb), 0.f);
    for (size_t i = 0; i < Ns.size(); ++i) {
      const int N = Ns[i];
      const mtf::TtBlock& q = p.blocks[i];
      W[i].resize(size_t(N) * N);  // W(r, j) at r * N + j
      F[i].resize(size_t(N));
      double wm = 0, bm = 0;
      for (auto& v : W[i]) v = float(G(rng) / std::sqrt(double(N))), wm = std::max(wm, std::fabs(v));
      for (int j = 0; j < N; ++j) F[i][size_t(j)] = cd(float(3 * G(rng)), float(G(rng)));
      for (int r = 0; r < N; ++r)
        for (int j = 0; j < N; ++j) {
          const double w = W[i][size_t(r) * N + j];
          bm = std::max(bm, std::fabs(w) * std::max(std::fabs(F[i][size_t(j)].real()), std::fabs(F[i][size_t(j)].imag())));
        }
      const float sa = p2scale(wm), sb = p2scale(bm);
      inv[i] = 1.f / (sa * sb);
      for (int r = 0; r < q.n_mt * mtf::kTcRows; ++r)
        for (int j = 0; j < q.n_kc * 64; ++j) {
          const float x = (r < N && j < N) ? float(W[i][size_t(r) * N + j]) * sa : 0.f;
          const float h = f16(x), l = f16(x - h);
          const int64_t tile = q.a_base + int64_t(r / mtf::kTcRows) * q.n_kc + j / 64;
          A[size_t(mtf::tc_tile_index(tile, 2, 0, r % mtf::kTcRows, j % 64))] = h;
          A[size_t(mtf::tc_tile_index(tile, 2, 1, r % mtf::kTcRows, j % 64))] = l;
        }
      for (int gr = 0; gr < q.n_nt * 128; ++gr)
        for (int j = 0; j < q.n_kc * 64; ++j) {
          const int c = gr / 2;
          float x = 0.f;
          if (c < N && j < N) {
            const cd fj = F[i][size_t(j)];
            x = float(W[i][size_t(c) * N + j]) * float((gr & 1) ? fj.imag() : fj.real()) * sb;
          }
          const float h = f16(x), l = f16(x - h);
          const int64_t chunk = q.b_base + int64_t(gr / 128) * q.n_kc + j / 64;
          B[size_t(mtf::tc_b_index(chunk, 0, gr % 128, j % 64, 128))] = h;
          B[size_t(mtf::tc_b_index(chunk, 1, gr % 128, j % 64, 128))] = l;
        }
    }
  }
  std::vector<std::vector<int>> cnt(Ns.size());
  std::vector<std::vector<cd>> T(Ns.size());
  for (size_t i = 0; i < Ns.size(); ++i) {
    cnt[i].assign(size_t(Ns[i]) * Ns[i], 0);
    T[i].assign(size_t(Ns[i]) * Ns[i], 0.0);
  }
  for (const mtf::TtUnit& u : p.units) {
    const mtf::TtBlock& q = p.blocks[size_t(u.blk)];
    const int64_t a0 = q.a_base + int64_t(u.mt) * q.n_kc, b0 = q.b_base + int64_t(u.nt) * q.n_kc;
    if (a0 + q.n_kc > p.n_a || b0 + q.n_kc > p.n_b) return std::printf("tt: index out of range\n"), 1;
    const int N = q.N;
    for (int rho = 0; rho < mtf::kTcRows; ++rho) {
      const int r = u.mt * mtf::kTcRows + rho;
      for (int cc = 0; cc < mtf::kTtCols; ++cc) {
        const int c = u.nt * mtf::kTtCols + cc;
        if (!(r < N && c < N && c >= r)) continue;
        float d[2] = {0.f, 0.f};
        if (emulate)
          for (int kc = 0; kc < q.n_kc; ++kc)
            for (int t = 0; t < 2; ++t)
              for (int e = 0; e < 64; ++e) {
                const float ah = A[size_t(mtf::tc_tile_index(a0 + kc, 2, 0, rho, e))];
                const float al = A[size_t(mtf::tc_tile_index(a0 + kc, 2, 1, rho, e))];
                const float bh = B[size_t(mtf::tc_b_index(b0 + kc, 0, 2 * cc + t, e, 128))];
                const float bl = B[size_t(mtf::tc_b_index(b0 + kc, 1, 2 * cc + t, e, 128))];
                d[t] += ah * bh + ah * bl + al * bh;
              }
        const cd o(d[0] * inv[size_t(u.blk)], d[1] * inv[size_t(u.blk)]);
        ++cnt[size_t(u.blk)][size_t(r) * N + c];
        T[size_t(u.blk)][size_t(r) * N + c] = o;
        if (c > r) {
          ++cnt[size_t(u.blk)][size_t(c) * N + r];
          T[size_t(u.blk)][size_t(c) * N + r] = o;
        }
      }
    }
  }
  for (auto& v : cnt)
    for (int x : v)
      if (x != 1) return std::printf("tt: an entry written %d times\n", x), 1;
  if (!emulate) return std::printf("tt: %zu blocks, %zu units, coverage ok\n", Ns.size(), p.units.size()), 0;
  double emax = 0;
  for (size_t i = 0; i < Ns.size(); ++i) {
    const int N = Ns[i];
    double tmax = 0, err = 0;
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {
        cd ex = 0;
        for (int j = 0; j < N; ++j) ex += W[i][size_t(r) * N + j] * F[i][size_t(j)] * W[i][size_t(c) * N + j];
        tmax = std::max(tmax, std::abs(ex));
        err = std::max(err, std::abs(ex - T[i][size_t(r) * N + c]));
      }
    emax = std::max(emax, err / tmax);
  }
  std::printf("tt: formation emulated, max entry error %.2e of the largest entry\n", emax);
  return emax < 4e-6 ? 0 : 1;
}

int main() {
  int f = 0;
  f += check_basis_layout();
  std::vector<int> cube4(65, 450);
  cube4[0] = 7200;
  f += check_plan(cube4, 152);
  f += check_plan({2178, 2178, 2178}, 152);
  f += check_plan({567, 45, 3}, 152);
  f += check_formulation();
  f += check_tt({2178, 2178, 2178}, false);
  f += check_tt(cube4, false);
  f += check_tt({200, 64, 129, 1}, true);
  return f;
}
