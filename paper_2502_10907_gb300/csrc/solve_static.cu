// mtf_solve_static: the GMRES solve of mtf_solve with every device buffer it
// needs (right-hand sides, Krylov basis, preconditioned directions, work
// vectors, Hessenberg columns, wave parameters) carved out of one fixed,
// file-scope device array instead of cudaMalloc.  It exists for callers that
// must not allocate device memory while they run -- code that executes under
// a custom or pre-reserved memory budget, or inside a host callback / service
// loop where a cudaMalloc could block on device synchronisation -- and who
// are willing to trade the size limit below for that.  Same algorithm as the
// FP64 path of mtf_solve (restarted flexible GMRES, right-preconditioned by
// block-OSRC when the system was assembled with it, CGS2, host Givens
// rotations) with its own simpler reduction kernels, so the two agree to
// rounding, not bit for bit.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <mutex>
#include <vector>

#include "common.h"

namespace mtf {

// capacity of the shared workspace, in doubles (16 MiB); every GPU that loads
// the library keeps this array resident until the process exits
constexpr size_t kStaticScratchDoubles = size_t(2) * 1024 * 1024;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

// kernels shared with the allocating solver (defined in solver.cu)
__global__ void k_dots(const double* __restrict__ V, const double* __restrict__ w, int64_t n, int ldv,
                       double* __restrict__ h, int ldh);
__global__ void k_axpy_multi(const double* __restrict__ V, const double* __restrict__ h, int j, int64_t n,
                             int ldv, int ldh, double sign, double* __restrict__ w, int nrhs);
__global__ void k_norm_scale(const double* __restrict__ w, int64_t n, double* __restrict__ nrm,
                             double* __restrict__ out, int64_t out_stride);
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                      int64_t n2);

// device address of g_static_scratch, looked up once per device (the host
// name of a __device__ array is a host-side stand-in, not a device address)
static std::mutex g_addr_mu;
static std::vector<double*> g_addr;

static double* scratch_address() {
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (int(g_addr.size()) <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    double* p = nullptr;
    MTF_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_static_scratch));
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

size_t static_solve_capacity() { return kStaticScratchDoubles; }

// doubles of workspace a solve of nrhs right-hand sides with restart m needs:
//   2 n nrhs (m + 4) + (6 m + 8) nrhs + 9 nrhs + 64, and with block-OSRC
//   another 2 n nrhs m (Z) + n nrhs (FP32 copy of the preconditioner input)
size_t static_solve_need(int64_t n, int nrhs, int m, bool pre) {
  const size_t n2 = size_t(n) * nrhs * 2;
  size_t need = n2 * size_t(m + 1) /*V*/ + 3 * n2 /*w, r, b*/ + size_t(2 * (m + 1) + 1) * nrhs * 2 /*h*/ +
                size_t(m + 1) * nrhs * 2 /*y*/ + size_t(nrhs) * 9 /*dirs, pols*/ + 64 /*alignment slack*/;
  if (pre) need += n2 * size_t(m) /*Z*/ + n2 / 2 /*r32*/;
  return need;
}

static inline unsigned nb(int64_t n, int t) { return unsigned((n + t - 1) / t); }

mtf_status solve_static(mtf_system sys, int nrhs, const double* dirs, const double* pols, double* x_dev,
                        mtf_solve_stats* st, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t n = sys->mesh->n_total;
  const int m = std::max(1, sys->opt.restart);
  MTF_REQUIRE(sys->opt.precision == MTF_PREC_FP64, MTF_ERR_ARG,
              "mtf_solve_static supports systems assembled with MTF_PREC_FP64 only");
  const bool pre = sys->opt.precond == MTF_PRECOND_OSRC;
  const size_t need = static_solve_need(n, nrhs, m, pre);
  MTF_REQUIRE(need <= kStaticScratchDoubles, MTF_ERR_ARG,
              "mtf_solve_static: the solve needs " + std::to_string(need) +
                  " doubles of workspace but the static workspace holds " +
                  std::to_string(kStaticScratchDoubles) +
                  " (16 MiB); lower nrhs or opt.restart, or use mtf_solve");
  double* base = scratch_address();
  // carve the workspace (offsets kept 32-byte aligned)
  size_t off = 0;
  auto take = [&](size_t count) {
    double* p = base + off;
    off += (count + 3) & ~size_t(3);
    return p;
  };
  const size_t n2 = size_t(n) * nrhs * 2;
  double* V = take(n2 * size_t(m + 1));
  double* w = take(n2);
  double* r = take(n2);
  double* b = take(n2);
  double* h = take(size_t(2 * (m + 1) + 1) * nrhs * 2);
  double* yd = take(size_t(m + 1) * nrhs * 2);
  double* d_dirs = take(size_t(nrhs) * 3);
  double* d_pols = take(size_t(nrhs) * 6);
  // flexible right preconditioning: z_j = P v_j in Z, the FP32 copy of v_j
  double* Z = pre ? take(n2 * size_t(m)) : nullptr;
  float* r32 = pre ? reinterpret_cast<float*>(take(n2 / 2)) : nullptr;
  // every call shares the array: clear the part this call uses
  MTF_CUDA(cudaMemsetAsync(base, 0, off * sizeof(double), s));
  MTF_CUDA(cudaMemcpyAsync(d_dirs, dirs, size_t(nrhs) * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyAsync(d_pols, pols, size_t(nrhs) * 6 * sizeof(double), cudaMemcpyHostToDevice, s));
  launch_rhs(sys, nrhs, d_dirs, d_pols, b, s);

  double* hA = h;
  double* hB = h + 2 * size_t(m + 1) * nrhs;
  double* hN = h + 4 * size_t(m + 1) * nrhs;
  std::vector<double> hhost(size_t(2 * (m + 1) + 1) * nrhs * 2);
  double* hostA = hhost.data();
  double* hostB = hhost.data() + 2 * size_t(m + 1) * nrhs;
  double* hostN = hhost.data() + 4 * size_t(m + 1) * nrhs;
  const int ldv = m + 1;
  const size_t vec_bytes = n2 * sizeof(double);
  using cd = std::complex<double>;

  std::vector<double> bnorm(nrhs), rel(nrhs, 1.0);
  MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(b, n, hN, w, n));
  MTF_CUDA(cudaMemcpyAsync(hostN, hN, size_t(nrhs) * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < nrhs; ++c) bnorm[c] = hostN[2 * c] > 0 ? hostN[2 * c] : 1.0;
  MTF_CUDA(cudaMemsetAsync(x_dev, 0, vec_bytes, s));

  std::vector<int> done(nrhs, 0), iters(nrhs, 0), jc(nrhs, 0), active(nrhs, 0);
  std::vector<cd> H(size_t(m + 1) * m * nrhs), g(size_t(m + 1) * nrhs), sn(size_t(m) * nrhs);
  std::vector<double> cs(size_t(m) * nrhs);
  std::vector<double> yhost(size_t(m + 1) * nrhs * 2);
  int restarts = 0, total = 0;
  bool first = true;
  const int max_iter = std::max(1, sys->opt.max_iter);
  const double tol = sys->opt.tol;
  mtf_status status = MTF_OK;
  while (true) {
    if (first) {
      MTF_CUDA(cudaMemcpyAsync(r, b, vec_bytes, cudaMemcpyDeviceToDevice, s));
    } else {
      launch_matvec(sys, x_dev, n, w, n, nrhs, s);
      MTF_LAUNCH(KID_SUB, s, k_sub<<<nb(int64_t(n2), 256), 256, 0, s>>>(b, w, r, int64_t(n2)));
    }
    first = false;
    MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(r, n, hN, V, int64_t(ldv) * n));
    MTF_CUDA(cudaMemcpyAsync(hostN, hN, size_t(nrhs) * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    bool all = true;
    for (int c = 0; c < nrhs; ++c) {
      rel[c] = hostN[2 * c] / bnorm[c];
      if (!std::isfinite(rel[c])) status = MTF_ERR_NAN;
      done[c] = rel[c] <= tol;
      all = all && done[c];
      jc[c] = 0;
      std::fill(g.begin() + size_t(c) * (m + 1), g.begin() + size_t(c + 1) * (m + 1), cd(0));
      g[size_t(c) * (m + 1)] = hostN[2 * c];
    }
    if (status != MTF_OK || all) break;
    if (total >= max_iter) {
      status = MTF_ERR_NOCONV;
      break;
    }
    ++restarts;
    for (int c = 0; c < nrhs; ++c) active[c] = !done[c];
    for (int j = 0; j < m && total < max_iter; ++j) {
      if (pre) {
        launch_osrc_apply_prepared(sys, V + 2 * size_t(j) * n, int64_t(ldv) * n, Z + 2 * size_t(j) * n,
                                   int64_t(m) * n, nrhs, r32, s);
        launch_matvec(sys, Z + 2 * size_t(j) * n, int64_t(m) * n, r, n, nrhs, s);
      } else {
        launch_matvec(sys, V + 2 * size_t(j) * n, int64_t(ldv) * n, r, n, nrhs, s);
      }
      dim3 gd(unsigned(j + 1), unsigned(nrhs));
      MTF_LAUNCH(KID_DOTS, s, k_dots<<<gd, 256, 0, s>>>(V, r, n, ldv, hA, m + 1));
      MTF_LAUNCH(KID_AXPY, s, k_axpy_multi<<<nb(n * nrhs, 256), 256, 0, s>>>(V, hA, j + 1, n, ldv, m + 1, -1.0, r, nrhs));
      MTF_LAUNCH(KID_DOTS, s, k_dots<<<gd, 256, 0, s>>>(V, r, n, ldv, hB, m + 1));
      MTF_LAUNCH(KID_AXPY, s, k_axpy_multi<<<nb(n * nrhs, 256), 256, 0, s>>>(V, hB, j + 1, n, ldv, m + 1, -1.0, r, nrhs));
      MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(r, n, hN, V + 2 * size_t(j + 1) * n, int64_t(ldv) * n));
      MTF_CUDA(cudaMemcpyAsync(hhost.data(), h, hhost.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      MTF_CUDA(cudaStreamSynchronize(s));
      ++total;
      bool all_done = true;
      for (int c = 0; c < nrhs; ++c) {
        if (!active[c]) continue;
        cd* Hc = &H[size_t(c) * (m + 1) * m + size_t(j) * (m + 1)];
        for (int q = 0; q <= j; ++q)
          Hc[q] = cd(hostA[2 * (size_t(c) * (m + 1) + q)] + hostB[2 * (size_t(c) * (m + 1) + q)],
                     hostA[2 * (size_t(c) * (m + 1) + q) + 1] + hostB[2 * (size_t(c) * (m + 1) + q) + 1]);
        Hc[j + 1] = cd(hostN[2 * c], 0.0);
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
        ++iters[c];
        const double est = std::abs(gc[j + 1]) / bnorm[c];
        if (!std::isfinite(est)) status = MTF_ERR_NAN;
        if (est <= tol * 0.5 || hostN[2 * c] == 0.0) active[c] = 0;
        all_done = all_done && !active[c];
      }
      if (status != MTF_OK || all_done) break;
    }
    if (status != MTF_OK) break;
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
    if (jmax > 0) {
      MTF_CUDA(cudaMemcpyAsync(yd, yhost.data(), yhost.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      // x += Z y (flexible) or V y
      MTF_LAUNCH(KID_AXPY, s, k_axpy_multi<<<nb(n * nrhs, 256), 256, 0, s>>>(pre ? Z : V, yd, jmax, n, pre ? m : ldv,
                                                                             m + 1, 1.0, x_dev, nrhs));
      MTF_CUDA(cudaStreamSynchronize(s));
    }
  }
  MTF_CUDA(cudaStreamSynchronize(s));
  if (st) {
    st->iterations = *std::max_element(iters.begin(), iters.end());
    st->restarts = restarts;
    st->refinements = 0;
    st->converged = status == MTF_OK;
    st->rel_residual = *std::max_element(rel.begin(), rel.end());
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

}  // namespace mtf

extern "C" mtf_status mtf_solve_static(mtf_system sys, int32_t nrhs, const double* dirs, const double* pols,
                                       void* x_out, mtf_solve_stats* stats, void* stream) {
  mtf_status st = MTF_OK;
  try {
    MTF_REQUIRE(sys && x_out && dirs && pols, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    for (int c = 0; c < nrhs; ++c) {
      const double* d = dirs + 3 * c;
      MTF_REQUIRE(std::fabs(std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - 1.0) < 1e-8, MTF_ERR_ARG,
                  "directions must be unit vectors");
    }
    st = mtf::solve_static(sys, nrhs, dirs, pols, static_cast<double*>(x_out), stats,
                           static_cast<cudaStream_t>(stream));
    if (st == MTF_ERR_NOCONV) mtf::set_last_error("GMRES did not reach the tolerance within max_iter");
    if (st == MTF_ERR_NAN) mtf::set_last_error("non-finite residual in GMRES");
  } catch (const mtf::Error& e) {
    mtf::set_last_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    mtf::set_last_error(e.what());
    return MTF_ERR_ARG;
  }
  return st;
}
