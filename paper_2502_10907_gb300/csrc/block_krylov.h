// Host side of block flexible GMRES (one Krylov space shared by all s
// right-hand sides of a solve): the deflating Cholesky factorisation that
// normalises a block of s new vectors, and the progressive Householder QR of
// the block upper-Hessenberg matrix with the residual estimates of every
// right-hand side and the final triangular solve.  Pure host C++ (no CUDA),
// so that it can be tested on its own.
//
// Notation.  Block step j produces W = M Z_j (n x s) orthogonalised against
// the basis V_0 .. V_j, with coefficients h = [V_0 .. V_j]^H W ((j+1) s x s),
// and W = V_{j+1} R_{j+1} with V_{j+1} orthonormal (deflated columns are zero)
// and R_{j+1} upper triangular.  Column block j of the Hessenberg matrix is
// [h; R_{j+1}] ((j+2) s x s).  Each column block is reduced to triangular
// form by s Householder reflectors acting on rows js + k .. (j+2)s - 1
// (reflector k of block j).  The right-hand side of the least-squares
// problem is E_1 S_0, S_0 the factor of the start block; after the
// reflectors of block j, rows (j+1)s .. (j+2)s - 1 of its column c hold the
// residual of right-hand side c.

#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstdlib>
#include <functional>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace mtf {

using cdouble = std::complex<double>;

// Cholesky factor of the Hermitian s x s Gram matrix G (column-major) of a
// block W, G = R^H R, skipping directions whose squared norm d_k after
// removing the earlier directions is at most tau^2 * ref[k] (ref[k] = a
// reference squared norm of column k, e.g. before orthogonalisation against
// the basis) or not positive: row k of R is then zero and column k of the
// normalised block is dropped (deflated).  T (s x s, column-major) receives
// the transform with V = W T: T[K, K] = R[K, K]^-1 on the kept index set K,
// zero elsewhere.  Returns the number of kept directions.
inline int deflating_cholesky(int s, const cdouble* G, const double* ref, double tau, cdouble* R, cdouble* T,
                              std::vector<int>& kept) {
  std::fill(R, R + size_t(s) * s, cdouble(0));
  std::fill(T, T + size_t(s) * s, cdouble(0));
  kept.assign(s, 0);
  for (int k = 0; k < s; ++k) {
    // R[i, k] for kept i < k
    for (int i = 0; i < k; ++i) {
      if (!kept[i]) continue;
      cdouble a = G[size_t(k) * s + i];
      for (int p = 0; p < i; ++p)
        if (kept[p]) a -= std::conj(R[size_t(i) * s + p]) * R[size_t(k) * s + p];
      R[size_t(k) * s + i] = a / R[size_t(i) * s + i];
    }
    double d = G[size_t(k) * s + k].real();
    for (int i = 0; i < k; ++i)
      if (kept[i]) d -= std::norm(R[size_t(k) * s + i]);
    const double lim = tau * tau * std::max(ref[k], 0.0);
    if (!(d > lim) || !(d > 0.0)) continue;  // deflated: column k keeps its projection R[i < k, k]
    kept[k] = 1;
    R[size_t(k) * s + k] = std::sqrt(d);
  }
  // rows of deflated indices are zero (their entries were never written)
  // T = R_KK^-1 by back substitution, column by column
  int nk = 0;
  for (int q = 0; q < s; ++q) {
    if (!kept[q]) continue;
    ++nk;
    T[size_t(q) * s + q] = 1.0 / R[size_t(q) * s + q];
    for (int i = q - 1; i >= 0; --i) {
      if (!kept[i]) continue;
      cdouble a = 0;
      for (int p = i + 1; p <= q; ++p)
        if (kept[p]) a += R[size_t(p) * s + i] * T[size_t(q) * s + p];
      T[size_t(q) * s + i] = -a / R[size_t(i) * s + i];
    }
  }
  return nk;
}

// Persistent host workers: run(n, f) calls f(i) for i in [0, n) on the
// workers and the calling thread and returns when all calls have finished
// and every worker is done with the task (so none can reach into the next
// one).  Workers poll for a new task for a short while (a block step's
// update follows the previous one within about a millisecond), then sleep on
// a condition variable.  One task at a time per pool.
class HostPool {
 public:
  explicit HostPool(int workers) {
    for (int t = 0; t < workers; ++t) th_.emplace_back([this] { loop(); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  HostPool(const HostPool&) = delete;
  HostPool& operator=(const HostPool&) = delete;

  void run(int n, const std::function<void(int)>& f) {
    fn_ = &f;
    n_ = n;
    next_.store(0, std::memory_order_relaxed);
    finished_.store(0, std::memory_order_relaxed);
    {
      std::lock_guard<std::mutex> lk(mu_);
      gen_.fetch_add(1, std::memory_order_release);  // publishes the task
    }
    cv_.notify_all();
    work();
    while (finished_.load(std::memory_order_acquire) < int(th_.size())) std::this_thread::yield();
  }

 private:
  void work() {
    for (int i = next_.fetch_add(1, std::memory_order_relaxed); i < n_; i = next_.fetch_add(1, std::memory_order_relaxed))
      (*fn_)(i);
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      uint64_t g = gen_.load(std::memory_order_acquire);
      for (int spin = 0; g == seen && spin < 4000; ++spin) {
        std::this_thread::yield();
        g = gen_.load(std::memory_order_acquire);
      }
      if (g == seen) {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
        g = gen_.load(std::memory_order_acquire);
      }
      seen = g;
      if (stop_) return;
      work();
      finished_.fetch_add(1, std::memory_order_release);
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::atomic<uint64_t> gen_{0};
  std::atomic<int> next_{0}, finished_{0};
  const std::function<void(int)>* fn_ = nullptr;
  int n_ = 0;
  bool stop_ = false;
};

struct BlockLSQ {
  int s = 0, m = 0;          // block size, maximum number of column blocks
  int k = 0;                 // column blocks added
  // reduced block columns: column block j is reduced in place in its slot of
  // the arena, (j + 2) s rows of s columns (column-major, leading dimension
  // (j + 2) s) at offset off[j]; rows 0 .. (j+1) s - 1 hold the triangular
  // factor.  The arena is allocated for m blocks once and reused by later
  // cycles (no per-step allocation; its pages are touched once).
  std::shared_ptr<cdouble> arena;
  size_t arena_len = 0;
  std::vector<size_t> off;
  // reflectors: block j, reflector kk: 2 s entries (top rows kk .. s-1 of
  // block row j, then the s rows of block row j + 1) and the scalar beta
  // (I - beta v v^H)
  std::vector<cdouble> refl;
  std::vector<double> beta;
  std::vector<cdouble> g;    // ldg x s, column-major: the least-squares right-hand sides
  size_t ldg = 0;
  std::vector<double> bnorm; // per right-hand side: reference norm of the estimates
  int threads = 1;
  mutable std::shared_ptr<HostPool> pool;  // threads - 1 workers, created with the first large update

  // f(c) for c in [0, n): on the pool when `big`, else on the calling thread
  void for_columns(int n, bool big, const std::function<void(int)>& f) const {
    if (!big || threads <= 1 || n <= 1) {
      for (int c = 0; c < n; ++c) f(c);
      return;
    }
    if (!pool) pool = std::make_shared<HostPool>(threads - 1);
    pool->run(n, f);
  }

  // S0: the start block's factor (s x s column-major), r = V_0 S0
  void init(int s_, int m_, const cdouble* S0, const double* base_norm) {
    s = s_;
    m = m_;
    k = 0;
    off.assign(size_t(m) + 1, 0);
    for (int j = 0; j < m; ++j) off[size_t(j) + 1] = off[size_t(j)] + size_t(j + 2) * s * s;
    if (off[size_t(m)] > arena_len) {
      arena.reset(static_cast<cdouble*>(std::malloc(off[size_t(m)] * sizeof(cdouble))), std::free);
      if (!arena) throw std::bad_alloc();
      arena_len = off[size_t(m)];
    }
    refl.assign(size_t(m) * s * 2 * s, cdouble(0));
    beta.assign(size_t(m) * s, 0.0);
    ldg = size_t(m + 2) * s;
    g.assign(ldg * s, cdouble(0));
    for (int c = 0; c < s; ++c)
      for (int i = 0; i < s; ++i) g[size_t(c) * ldg + i] = S0[size_t(c) * s + i];
    bnorm.assign(s, 1.0);
    for (int c = 0; c < s; ++c) bnorm[c] = base_norm[c] > 0 ? base_norm[c] : 1.0;
    const unsigned hw = std::thread::hardware_concurrency();
    threads = int(std::max(1u, std::min(hw, 16u)));
  }

  // apply reflector (j, kk) to one column x (rows j s + kk .. (j + 2) s - 1)
  // (written on the (re, im) doubles of the complex arrays, with two
  // independent partial sums, which the compiler keeps in registers)
  inline void apply_reflector(int j, int kk, cdouble* x) const {
    const double b = beta[size_t(j) * s + kk];
    if (b == 0.0) return;
    const double* v = reinterpret_cast<const double*>(&refl[(size_t(j) * s + kk) * 2 * s]);
    double* top = reinterpret_cast<double*>(x + size_t(j) * s + kk);
    const int len = 2 * s - kk;
    double ar0 = 0, ai0 = 0, ar1 = 0, ai1 = 0;  // a = sum conj(v_t) x_t
    int t = 0;
    for (; t + 1 < len; t += 2) {
      const double vr0 = v[2 * t], vi0 = v[2 * t + 1], xr0 = top[2 * t], xi0 = top[2 * t + 1];
      const double vr1 = v[2 * t + 2], vi1 = v[2 * t + 3], xr1 = top[2 * t + 2], xi1 = top[2 * t + 3];
      ar0 += vr0 * xr0 + vi0 * xi0;
      ai0 += vr0 * xi0 - vi0 * xr0;
      ar1 += vr1 * xr1 + vi1 * xi1;
      ai1 += vr1 * xi1 - vi1 * xr1;
    }
    if (t < len) {
      ar0 += v[2 * t] * top[2 * t] + v[2 * t + 1] * top[2 * t + 1];
      ai0 += v[2 * t] * top[2 * t + 1] - v[2 * t + 1] * top[2 * t];
    }
    const double ar = (ar0 + ar1) * b, ai = (ai0 + ai1) * b;
    for (t = 0; t < len; ++t) {  // x -= v a
      const double vr = v[2 * t], vi = v[2 * t + 1];
      top[2 * t] -= vr * ar - vi * ai;
      top[2 * t + 1] -= vr * ai + vi * ar;
    }
  }

  // apply reflector (j, kk) to NC columns at once (one pass over v, NC
  // independent chains)
  template <int NC>
  inline void apply_reflector_cols(int j, int kk, cdouble* const* xs) const {
    const double b = beta[size_t(j) * s + kk];
    if (b == 0.0) return;
    const double* v = reinterpret_cast<const double*>(&refl[(size_t(j) * s + kk) * 2 * s]);
    double* p[NC];
    for (int c = 0; c < NC; ++c) p[c] = reinterpret_cast<double*>(xs[c] + size_t(j) * s + kk);
    const int len = 2 * s - kk;
    double ar[NC], ai[NC];
    for (int c = 0; c < NC; ++c) ar[c] = ai[c] = 0.0;
    for (int t = 0; t < len; ++t) {
      const double vr = v[2 * t], vi = v[2 * t + 1];
      for (int c = 0; c < NC; ++c) {
        ar[c] += vr * p[c][2 * t] + vi * p[c][2 * t + 1];
        ai[c] += vr * p[c][2 * t + 1] - vi * p[c][2 * t];
      }
    }
    for (int c = 0; c < NC; ++c) {
      ar[c] *= b;
      ai[c] *= b;
    }
    for (int t = 0; t < len; ++t) {
      const double vr = v[2 * t], vi = v[2 * t + 1];
      for (int c = 0; c < NC; ++c) {
        p[c][2 * t] -= vr * ar[c] - vi * ai[c];
        p[c][2 * t + 1] -= vr * ai[c] + vi * ar[c];
      }
    }
  }

  // earlier blocks' reflectors on the columns [c0, c0 + n) of x (column
  // stride rows), NC at a time
  template <int NC>
  void earlier_reflectors(int j, cdouble* col, size_t rows, int c0, int n) const {
    int c = c0;
    for (; c + NC <= c0 + n; c += NC) {
      cdouble* xs[NC];
      for (int q = 0; q < NC; ++q) xs[q] = col + size_t(c + q) * rows;
      for (int q = 0; q < j; ++q)
        for (int kk = 0; kk < s; ++kk) apply_reflector_cols<NC>(q, kk, xs);
    }
    for (; c < c0 + n; ++c)
      for (int q = 0; q < j; ++q)
        for (int kk = 0; kk < s; ++kk) apply_reflector(q, kk, col + size_t(c) * rows);
  }

  // Add column block j = k: h (nrows_h = j + 1 blocks of s rows x s,
  // column-major, leading dimension nrows_h s) on the basis blocks
  // 0 .. j and the upper-triangular R (s x s) on block j + 1.  est[c]
  // receives the relative residual estimate of right-hand side c.  Returns
  // false when m blocks are stored or nrows_h != j + 1.
  bool add_block(const cdouble* h, int nrows_h, const cdouble* R, double* est) {
    if (k >= m) return false;
    const int j = k;
    const int b = nrows_h - j;
    if (b != 1) return false;
    const size_t rows = size_t(nrows_h + 1) * s, hr = size_t(nrows_h) * s;
    cdouble* col = arena.get() + off[size_t(j)];  // this block's slot, leading dimension rows
    for (int c = 0; c < s; ++c) {
      cdouble* x = &col[size_t(c) * rows];
      for (size_t i = 0; i < hr; ++i) x[i] = h[size_t(c) * hr + i];
      for (int i = 0; i < s; ++i) x[hr + i] = R[size_t(c) * s + i];
    }
    // earlier reflectors, column by column (independent columns)
    const long work = long(j) * s * (2 * s) * s;
    // (columns in groups: one pass over the stored reflectors serves 2, or 4
    // for blocks of 32 columns or more)
    const int G = s >= 32 ? 4 : 2;
    for_columns((s + G - 1) / G, work > 200000, [&](int cg) {
      const int c0 = cg * G, n = std::min(G, s - c0);
      if (G == 4) earlier_reflectors<4>(j, col, rows, c0, n);
      else earlier_reflectors<2>(j, col, rows, c0, n);
    });
    // reflectors of this block: column kk, rows j s + kk .. (j + 1 + b) s - 1.
    // Wide blocks (32 columns or more) take them in panels of 8 columns: a
    // panel's reflectors are formed and applied within the panel, then
    // applied to the columns to its right on the pool (each column still
    // sees the reflectors in order)
    const bool wide = s >= 32 && threads > 1;
    const int P = wide ? 8 : s;
    for (int k0 = 0; k0 < s; k0 += P) {
      const int k1 = std::min(s, k0 + P);
      for (int kk = k0; kk < k1; ++kk) {
        cdouble* x = &col[size_t(kk) * rows] + size_t(j) * s + kk;
        cdouble* v = &refl[(size_t(j) * s + kk) * 2 * s];
        const int len = 2 * s - kk;
        double nrm2 = 0;
        for (int t = 0; t < len; ++t) nrm2 += std::norm(x[t]);
        const double nrm = std::sqrt(nrm2);
        if (nrm == 0.0) {
          beta[size_t(j) * s + kk] = 0.0;
          continue;
        }
        const cdouble x0 = x[0];
        const double ax0 = std::abs(x0);
        const cdouble ph = ax0 > 0 ? x0 / ax0 : cdouble(1.0);
        const cdouble alpha = -ph * nrm;  // x -> alpha e_0
        for (int t = 0; t < len; ++t) v[t] = x[t];
        for (int t = len; t < 2 * s; ++t) v[t] = 0;
        v[0] -= alpha;
        double vn2 = 0;
        for (int t = 0; t < len; ++t) vn2 += std::norm(v[t]);
        beta[size_t(j) * s + kk] = vn2 > 0 ? 2.0 / vn2 : 0.0;
        for (int c = kk; c < k1; ++c) apply_reflector(j, kk, &col[size_t(c) * rows]);
      }
      if (k1 < s)
        for_columns(s - k1, wide, [&](int i) {
          cdouble* x = &col[size_t(k1 + i) * rows];
          for (int kk = k0; kk < k1; ++kk) apply_reflector(j, kk, x);
        });
    }
    // the reduced block stays in its slot (rows 0 .. (j+1) s - 1); the
    // least-squares right-hand sides take the block's reflectors
    for_columns(s, wide, [&](int c) {
      for (int kk = 0; kk < s; ++kk) apply_reflector(j, kk, &g[size_t(c) * ldg]);
    });
    ++k;
    for (int c = 0; c < s; ++c) {
      double r2 = 0;
      for (int i = 0; i < s; ++i) r2 += std::norm(g[size_t(c) * ldg + size_t(k) * s + i]);
      est[c] = std::sqrt(r2) / bnorm[c];
    }
    return true;
  }

  // Y (k s x s, column-major, ld k s): the block coefficients minimising the
  // residual of every right-hand side.  Diagonal entries below eps times the
  // largest one (deflated or breakdown directions) give zero coefficients.
  void solve(std::vector<cdouble>& Y) const {
    const size_t n = size_t(k) * s;
    Y.assign(n * s, cdouble(0));
    double dmax = 0;
    for (size_t i = 0; i < n; ++i) dmax = std::max(dmax, std::abs(diag(i)));
    const double eps = 1e-13 * dmax;
    for_columns(s, n * n * s > 4000000, [&](int c) {
      cdouble* y = &Y[size_t(c) * n];
      for (size_t i = 0; i < n; ++i) y[i] = g[size_t(c) * ldg + i];
      for (size_t ii = n; ii-- > 0;) {
        const cdouble d = diag(ii);
        if (std::abs(d) <= eps) {
          y[ii] = 0;
          continue;
        }
        y[ii] /= d;
        // subtract column ii's entries above the diagonal
        const int jb = int(ii / s), cc = int(ii % s);
        const cdouble* colp = arena.get() + off[size_t(jb)] + size_t(cc) * (jb + 2) * s;
        for (size_t t = 0; t < ii; ++t) y[t] -= colp[t] * y[ii];
      }
    });
  }

  cdouble diag(size_t i) const {
    const int jb = int(i / s), cc = int(i % s);
    return arena.get()[off[size_t(jb)] + size_t(cc) * (jb + 2) * s + i];
  }
};

}  // namespace mtf
