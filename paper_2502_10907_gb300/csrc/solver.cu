// Restarted flexible GMRES for M u = b (Sec. 5.3: relative tolerance and an
// iteration cap), batched over right-hand sides: every right-hand side has its
// own Krylov basis, all of them advance together so that each operator apply
// is one multi-column matvec.  Orthogonalisation is classical Gram-Schmidt
// applied twice (CGS2) in FP64 on the device; the small Hessenberg least-
// squares problems (Givens rotations) run on the host from the (j+2) new
// Hessenberg entries per right-hand side copied back each iteration.  A
// restart cycle ends on convergence of every right-hand side, on the restart
// length or on the iteration cap; each cycle starts from the true residual
// b - M x, which is also the stopping test.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <complex>

#include "common.h"

namespace mtf {

using cd = std::complex<double>;

struct GmresWork {
  int nrhs = 0, m = 0;
  int64_t n = 0;
  DevBuf<double> V, Z, w, r, b, y;
  DevBuf<double> h;  // [hA (m+1) x nrhs][hB (m+1) x nrhs][norm nrhs] complex
  double* h_host = nullptr;
  ~GmresWork() {
    if (h_host) cudaFreeHost(h_host);
  }
};

void destroy_gmres(GmresWork* w) { delete w; }

// h[c*(ldh) + i] = <V_i^c, w^c> = sum conj(V) w  for i < j, one CTA per (i, c)
__global__ void __launch_bounds__(256) k_dots(const double* __restrict__ V, const double* __restrict__ w,
                                              int64_t n, int ldv, double* __restrict__ h, int ldh) {
  const int i = blockIdx.x, c = blockIdx.y;
  const double2* v = reinterpret_cast<const double2*>(V) + (int64_t(c) * ldv + i) * n;
  const double2* x = reinterpret_cast<const double2*>(w) + int64_t(c) * n;
  double sr = 0, si = 0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double2 a = v[k], b = x[k];
    sr += a.x * b.x + a.y * b.y;
    si += a.x * b.y - a.y * b.x;
  }
  __shared__ double red[2][8];
  for (int s = 16; s > 0; s >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, s);
    si += __shfl_xor_sync(0xffffffffu, si, s);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) {
      a += red[0][q];
      b += red[1][q];
    }
    h[2 * (int64_t(c) * ldh + i)] = a;
    h[2 * (int64_t(c) * ldh + i) + 1] = b;
  }
}

// w^c += sign * sum_{i<j} V_i^c h_i^c
__global__ void k_axpy_multi(const double* __restrict__ V, const double* __restrict__ h, int j, int64_t n,
                             int ldv, int ldh, double sign, double* __restrict__ w, int nrhs) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int c = int(t / n);
  const int64_t k = t % n;
  const double2* v = reinterpret_cast<const double2*>(V) + int64_t(c) * ldv * n + k;
  const double* hc = h + 2 * int64_t(c) * ldh;
  double sr = 0, si = 0;
  for (int i = 0; i < j; ++i) {
    const double2 a = v[int64_t(i) * n];
    const double hr = hc[2 * i], hi = hc[2 * i + 1];
    sr += a.x * hr - a.y * hi;
    si += a.x * hi + a.y * hr;
  }
  double2* x = reinterpret_cast<double2*>(w) + int64_t(c) * n + k;
  double2 o = *x;
  o.x += sign * sr;
  o.y += sign * si;
  *x = o;
}

// nrm[c] = ||w^c||, out^c = w^c / nrm[c] (zero if nrm is 0); one CTA per c
__global__ void __launch_bounds__(1024) k_norm_scale(const double* __restrict__ w, int64_t n,
                                                      double* __restrict__ nrm, double* __restrict__ out,
                                                      int64_t out_stride) {
  const int c = blockIdx.x;
  const double2* x = reinterpret_cast<const double2*>(w) + int64_t(c) * n;
  double s = 0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += x[k].x * x[k].x + x[k].y * x[k].y;
  __shared__ double red[32];
  __shared__ double tot;
  for (int q = 16; q > 0; q >>= 1) s += __shfl_xor_sync(0xffffffffu, s, q);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) a += red[q];
    tot = sqrt(a);
    nrm[2 * c] = tot;
    nrm[2 * c + 1] = 0.0;
  }
  __syncthreads();
  const double inv = tot > 0 ? 1.0 / tot : 0.0;
  double2* o = reinterpret_cast<double2*>(out) + int64_t(c) * out_stride;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) o[k] = make_double2(x[k].x * inv, x[k].y * inv);
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                      int64_t n2) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n2) out[t] = a[t] - b[t];
}

static inline unsigned nblk(int64_t n, int t) { return unsigned((n + t - 1) / t); }

// Segmented kernels of the batched Arnoldi step: the row range is cut into
// segments of kSeg entries so that every step keeps the whole GPU busy;
// per-segment partial sums are accumulated with FP64 atomics (the
// accumulators are cleared before each use).
constexpr int kSeg = 2048;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int s = 16; s > 0; s >>= 1) t += __shfl_xor_sync(0xffffffffu, t, s);
  }
  return t;  // valid in thread 0
}

// h[c*ldh + i] += sum_k conj(V_i^c[k]) w^c[k] over one segment of length seg;
// grid (segments, i, c)
__global__ void __launch_bounds__(256) k_dots_seg(const double* __restrict__ V, const double* __restrict__ w,
                                                  int64_t n, int ldv, double* __restrict__ h, int ldh, int64_t seg) {
  const int i = blockIdx.y, c = blockIdx.z;
  const int64_t k0 = int64_t(blockIdx.x) * seg;
  const int64_t k1 = min(n, k0 + seg);
  const double2* v = reinterpret_cast<const double2*>(V) + (int64_t(c) * ldv + i) * n;
  const double2* x = reinterpret_cast<const double2*>(w) + int64_t(c) * n;
  double sr = 0, si = 0;
#pragma unroll 8
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double2 a = v[k], b = x[k];
    sr += a.x * b.x + a.y * b.y;
    si += a.x * b.y - a.y * b.x;
  }
  __shared__ double red[32];
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  if (threadIdx.x == 0) {
    atomicAdd(h + 2 * (int64_t(c) * ldh + i), sr);
    atomicAdd(h + 2 * (int64_t(c) * ldh + i) + 1, si);
  }
}

// h[c*ldh + i] += sum_{k in segment} conj(V_i^c[k]) w^c[k]: CTA = one column
// segment (<= 2048 entries of w staged in shared memory) x 16 basis vectors
// (2 per warp, interleaved for 16 loads in flight); grid (segments,
// ceil(rows/16), c).
__global__ void __launch_bounds__(256) k_dots_stage(const double* __restrict__ V, const double* __restrict__ w,
                                                    int64_t n, int ldv, int rows, double* __restrict__ h, int ldh,
                                                    int64_t seg) {
  extern __shared__ double2 ws[];
  const int c = blockIdx.z;
  const int64_t k0 = int64_t(blockIdx.x) * seg;
  const int len = int(min(n, k0 + seg) - k0);
  const double2* wc = reinterpret_cast<const double2*>(w) + int64_t(c) * n + k0;
  for (int t = threadIdx.x; t < len; t += blockDim.x) ws[t] = wc[t];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * 16 + warp * 2;
  if (i0 >= rows) return;
  const bool two = i0 + 1 < rows;
  const double2* v0 = reinterpret_cast<const double2*>(V) + (int64_t(c) * ldv + i0) * n + k0;
  const double2* v1 = two ? v0 + n : v0;
  double r0 = 0, q0 = 0, r1 = 0, q1 = 0;
#pragma unroll 8
  for (int t = lane; t < len; t += 32) {
    const double2 a = v0[t], b = v1[t], x = ws[t];
    r0 += a.x * x.x + a.y * x.y;
    q0 += a.x * x.y - a.y * x.x;
    r1 += b.x * x.x + b.y * x.y;
    q1 += b.x * x.y - b.y * x.x;
  }
#pragma unroll
  for (int s2 = 16; s2 > 0; s2 >>= 1) {
    r0 += __shfl_xor_sync(0xffffffffu, r0, s2);
    q0 += __shfl_xor_sync(0xffffffffu, q0, s2);
    r1 += __shfl_xor_sync(0xffffffffu, r1, s2);
    q1 += __shfl_xor_sync(0xffffffffu, q1, s2);
  }
  if (lane == 0) {
    atomicAdd(h + 2 * (int64_t(c) * ldh + i0), r0);
    atomicAdd(h + 2 * (int64_t(c) * ldh + i0) + 1, q0);
    if (two) {
      atomicAdd(h + 2 * (int64_t(c) * ldh + i0 + 1), r1);
      atomicAdd(h + 2 * (int64_t(c) * ldh + i0 + 1) + 1, q1);
    }
  }
}

static void launch_dots(const double* V, const double* w, int64_t n, int ldv, int rows, double* h, int ldh, int nrhs,
                        cudaStream_t s) {
  const int64_t rg = (rows + 15) / 16;
  const int64_t minseg = (n + 2047) / 2048;
  const int64_t nseg = std::max<int64_t>(minseg, std::min<int64_t>((n + 511) / 512, 1200 / (rg * nrhs)));
  const int64_t seg = (n + nseg - 1) / nseg;
  dim3 g{unsigned(nseg), unsigned(rg), unsigned(nrhs)};
  MTF_LAUNCH(KID_DOTS, s, k_dots_stage<<<g, 256, size_t(seg) * sizeof(double2), s>>>(V, w, n, ldv, rows, h, ldh, seg));
}

// w^c -= sum_{i<j} V_i^c h_i^c ; optionally ss[c] += ||w^c||^2 (after update).
// CTA = 32 consecutive rows x 8 groups of basis vectors (i = g mod 8), the
// group partial sums combined in shared memory; grid (ceil(n/32), c).
__global__ void __launch_bounds__(256) k_axpy_grp(const double* __restrict__ V, const double* __restrict__ h, int j,
                                                  int64_t n, int ldv, int ldh, double sign, double* __restrict__ w,
                                                  double* __restrict__ ss) {
  const int c = blockIdx.y;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t k = int64_t(blockIdx.x) * 32 + lane;
  __shared__ double2 part[8][32];
  __shared__ double red[32];
  extern __shared__ double2 hs[];  // h of this rhs (j entries)
  const double2* hc = reinterpret_cast<const double2*>(h) + int64_t(c) * ldh;
  for (int t = threadIdx.x; t < j; t += blockDim.x) hs[t] = hc[t];
  __syncthreads();
  double sr = 0, si = 0;
  if (k < n) {
    const double2* v = reinterpret_cast<const double2*>(V) + int64_t(c) * ldv * n + k;
#pragma unroll 8
    for (int i = grp; i < j; i += 8) {
      const double2 a = v[int64_t(i) * n];
      const double2 hv = hs[i];
      sr += a.x * hv.x - a.y * hv.y;
      si += a.x * hv.y + a.y * hv.x;
    }
  }
  part[grp][lane] = make_double2(sr, si);
  __syncthreads();
  double sq = 0;
  if (grp == 0 && k < n) {
    double tr = 0, ti = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      tr += part[g][lane].x;
      ti += part[g][lane].y;
    }
    double2* x = reinterpret_cast<double2*>(w) + int64_t(c) * n + k;
    double2 o = *x;
    o.x += sign * tr;
    o.y += sign * ti;
    *x = o;
    sq = o.x * o.x + o.y * o.y;
  }
  if (ss) {
    if (grp == 0) {
      for (int s2 = 16; s2 > 0; s2 >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s2);
      if (lane == 0) atomicAdd(ss + c, sq);
    }
  }
  (void)red;
}

__global__ void __launch_bounds__(256) k_axpy_sq(const double* __restrict__ V, const double* __restrict__ h, int j,
                                                 int64_t n, int ldv, int ldh, double sign, double* __restrict__ w,
                                                 double* __restrict__ ss) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double sq = 0;
  if (k < n) {
    const double2* v = reinterpret_cast<const double2*>(V) + int64_t(c) * ldv * n + k;
    const double* hc = h + 2 * int64_t(c) * ldh;
    double sr = 0, si = 0;
#pragma unroll 8
    for (int i = 0; i < j; ++i) {
      const double2 a = v[int64_t(i) * n];
      const double hr = hc[2 * i], hi = hc[2 * i + 1];
      sr += a.x * hr - a.y * hi;
      si += a.x * hi + a.y * hr;
    }
    double2* x = reinterpret_cast<double2*>(w) + int64_t(c) * n + k;
    double2 o = *x;
    o.x += sign * sr;
    o.y += sign * si;
    *x = o;
    sq = o.x * o.x + o.y * o.y;
  }
  if (ss) {
    __shared__ double red[32];
    sq = block_sum(sq, red);
    if (threadIdx.x == 0) atomicAdd(ss + c, sq);
  }
}

// ss[c] += ||w^c||^2
__global__ void __launch_bounds__(256) k_sqnorm(const double* __restrict__ w, int64_t n, double* __restrict__ ss) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double sq = 0;
  if (k < n) {
    const double2 a = reinterpret_cast<const double2*>(w)[int64_t(c) * n + k];
    sq = a.x * a.x + a.y * a.y;
  }
  __shared__ double red[32];
  sq = block_sum(sq, red);
  if (threadIdx.x == 0) atomicAdd(ss + c, sq);
}

// out^c = w^c / sqrt(ss[c]) (zero if 0); nrm[c] = (sqrt(ss[c]), 0)
__global__ void __launch_bounds__(256) k_scale(const double* __restrict__ w, int64_t n, const double* __restrict__ ss,
                                               double* __restrict__ nrm, double* __restrict__ out,
                                               int64_t out_stride) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const double t = sqrt(ss[c]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    nrm[2 * c] = t;
    nrm[2 * c + 1] = 0.0;
  }
  if (k >= n) return;
  const double inv = t > 0 ? 1.0 / t : 0.0;
  const double2 a = reinterpret_cast<const double2*>(w)[int64_t(c) * n + k];
  reinterpret_cast<double2*>(out)[int64_t(c) * out_stride + k] = make_double2(a.x * inv, a.y * inv);
}

// One restarted GMRES solve of M x = b (x starts at 0) with the given matvec
// flavour.  Per right-hand side: iters[c] += inner iterations, rel[c] = final
// true relative residual (w.r.t. the same flavour).
static mtf_status gmres_core(mtf_system sys, int nrhs, const double* b_dev, double* x_dev, int mvkind,
                             double tol, int max_iter, std::vector<int>& iters, int& restarts,
                             std::vector<double>& rel, cudaStream_t s) {
  mtf_mesh msh = sys->mesh;
  const int64_t n = msh->n_total;
  const int m = std::max(1, sys->opt.restart);
  GmresWork& G = *sys->gw;
  double* hA = G.h.p;
  double* hB = G.h.p + 2 * size_t(m + 1) * nrhs;
  double* hN = G.h.p + 4 * size_t(m + 1) * nrhs;
  double* hostA = G.h_host;
  double* hostB = G.h_host + 2 * size_t(m + 1) * nrhs;
  double* hostN = G.h_host + 4 * size_t(m + 1) * nrhs;
  const int ldv = m + 1;
  const size_t vec_bytes = size_t(n) * nrhs * 2 * sizeof(double);

  std::vector<double> bnorm(nrhs);
  MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(b_dev, n, hN, G.w.p, n));
  MTF_CUDA(cudaMemcpyAsync(hostN, hN, size_t(nrhs) * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < nrhs; ++c) bnorm[c] = hostN[2 * c] > 0 ? hostN[2 * c] : 1.0;
  MTF_CUDA(cudaMemsetAsync(x_dev, 0, vec_bytes, s));

  std::vector<int> done(nrhs, 0), jc(nrhs, 0);
  std::vector<cd> H(size_t(m + 1) * m * nrhs), g(size_t(m + 1) * nrhs), sn(size_t(m) * nrhs);
  std::vector<double> cs(size_t(m) * nrhs);
  std::vector<double> yhost(size_t(m + 1) * nrhs * 2);
  int total = 0;
  bool first = true;
  mtf_status status = MTF_OK;
  const bool pre = sys->opt.precond == MTF_PRECOND_OSRC;
  if (pre && G.Z.n != size_t(m) * n * nrhs * 2) G.Z.alloc(size_t(m) * n * nrhs * 2);
  while (true) {
    // true residual r = b - M x and its norm; V_0 = r / ||r||
    if (first) {
      MTF_CUDA(cudaMemcpyAsync(G.r.p, b_dev, vec_bytes, cudaMemcpyDeviceToDevice, s));
    } else {
      launch_matvec_kind(sys, mvkind, x_dev, n, G.w.p, n, nrhs, s);
      MTF_LAUNCH(KID_SUB, s, k_sub<<<nblk(n * nrhs * 2, 256), 256, 0, s>>>(b_dev, G.w.p, G.r.p, n * nrhs * 2));
    }
    first = false;
    MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(G.r.p, n, hN, G.V.p, int64_t(ldv) * n));
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
    if (status != MTF_OK) break;
    if (all) break;
    if (total >= max_iter) {
      status = MTF_ERR_NOCONV;
      break;
    }
    ++restarts;
    std::vector<int> active(nrhs);
    for (int c = 0; c < nrhs; ++c) active[c] = !done[c];
    for (int j = 0; j < m && total < max_iter; ++j) {
      // flexible right preconditioning: z_j = P v_j, w = M z_j
      if (pre) {
        launch_osrc_apply(sys, G.V.p + 2 * size_t(j) * n, int64_t(ldv) * n, G.Z.p + 2 * size_t(j) * n,
                          int64_t(m) * n, nrhs, s);
        launch_matvec_kind(sys, mvkind, G.Z.p + 2 * size_t(j) * n, int64_t(m) * n, G.r.p, n, nrhs, s);
      } else {
        launch_matvec_kind(sys, mvkind, G.V.p + 2 * size_t(j) * n, int64_t(ldv) * n, G.r.p, n, nrhs, s);
      }
      // CGS2: h_A = V^H w, w -= V h_A, h_B = V^H w, w -= V h_B (with ||w||^2)
      MTF_CUDA(cudaMemsetAsync(G.h.p, 0, G.h.n * sizeof(double), s));
      // segments per dot so that ~1200 CTAs run whatever j is
      const int64_t nseg = std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024,
                                                                  1200 / (int64_t(j + 1) * nrhs)));
      const int64_t seg = (n + nseg - 1) / nseg;
      dim3 gd(unsigned(nseg), unsigned(j + 1), unsigned(nrhs));
      dim3 ga(nblk(n, 256), unsigned(nrhs));
      dim3 gg(nblk(n, 32), unsigned(nrhs));
      double* ss = hN + 2 * nrhs;  // sum of squares scratch after the norms
      const size_t hsm = size_t(j + 1) * sizeof(double2);
      (void)gd;
      launch_dots(G.V.p, G.r.p, n, ldv, j + 1, hA, m + 1, nrhs, s);
      MTF_LAUNCH(KID_AXPY, s, k_axpy_grp<<<gg, 256, hsm, s>>>(G.V.p, hA, j + 1, n, ldv, m + 1, -1.0, G.r.p, nullptr));
      launch_dots(G.V.p, G.r.p, n, ldv, j + 1, hB, m + 1, nrhs, s);
      MTF_LAUNCH(KID_AXPY, s, k_axpy_grp<<<gg, 256, hsm, s>>>(G.V.p, hB, j + 1, n, ldv, m + 1, -1.0, G.r.p, ss));
      // v_{j+1} = w / ||w||
      MTF_LAUNCH(KID_NORM, s, k_scale<<<ga, 256, 0, s>>>(G.r.p, n, ss, hN, G.V.p + 2 * size_t(j + 1) * n, int64_t(ldv) * n));
      MTF_CUDA(cudaMemcpyAsync(G.h_host, G.h.p, G.h.n * sizeof(double), cudaMemcpyDeviceToHost, s));
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
        // previous rotations
        for (int q = 0; q < j; ++q) {
          const double cq = cs[size_t(c) * m + q];
          const cd sq = sn[size_t(c) * m + q];
          const cd t = cq * Hc[q] + sq * Hc[q + 1];
          Hc[q + 1] = -std::conj(sq) * Hc[q] + cq * Hc[q + 1];
          Hc[q] = t;
        }
        // new rotation zeroing H[j+1, j]
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
    // x += V y, y = R^{-1} g per right-hand side
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
      MTF_CUDA(cudaMemcpyAsync(G.y.p, yhost.data(), yhost.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      // x += Z y (flexible) or V y
      MTF_LAUNCH(KID_AXPY, s, k_axpy_grp<<<dim3(nblk(n, 32), unsigned(nrhs)), 256, size_t(jmax) * sizeof(double2), s>>>(
          pre ? G.Z.p : G.V.p, G.y.p, jmax, n, pre ? m : ldv, m + 1, 1.0, x_dev, nullptr));
      MTF_CUDA(cudaStreamSynchronize(s));  // yhost is reused next cycle
    }
  }
  return status;
}

// Fewest right-hand sides for which the block cycle is used.  With 2 waves
// of one incidence direction (the split sphere) the block space needed as
// many steps as each single space (437 against 440) and its per-step host
// synchronisation made the solve slower; with 16 waves of 8 directions (the
// 4 x 4 x 4 cube) it needed 838 block steps where single spaces needed
// about 6,000 iterations.
constexpr int kBlockMinRhs = 4;

__global__ void k_add(double* __restrict__ x, const double* __restrict__ d, int64_t n2) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n2) x[t] += d[t];
}

mtf_status solve(mtf_system sys, int nrhs, const double* b_dev, double* x_dev, mtf_solve_stats* st,
                 cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  sys->t_launch = sys->t_lsq = sys->t_wait = 0;
  mtf_mesh msh = sys->mesh;
  const int64_t n = msh->n_total;
  const int m = std::max(1, sys->opt.restart);
  if (!sys->gw) sys->gw = new GmresWork();
  GmresWork& G = *sys->gw;
  const bool mixed = sys->opt.precision != MTF_PREC_FP64;
  sys->learned_active = false;  // the learned correction runs in the mixed path only
  if (G.nrhs != nrhs || G.m != m || G.n != n) {
    G.V.alloc(size_t(m + 1) * n * nrhs * 2);
    G.w.alloc(size_t(n) * nrhs * 2);
    G.r.alloc(size_t(n) * nrhs * 2);
    G.y.alloc(size_t(m + 1) * nrhs * 2);
    G.h.alloc(size_t(2 * (m + 1) + 2) * nrhs * 2);
    if (G.h_host) cudaFreeHost(G.h_host);
    G.h_host = nullptr;
    MTF_CUDA(cudaMallocHost(&G.h_host, G.h.n * sizeof(double)));
    G.nrhs = nrhs;
    G.m = m;
    G.n = n;
  }
  std::vector<int> iters(nrhs, 0);
  std::vector<double> rel(nrhs, 1.0);
  int restarts = 0, refinements = 0;
  const int max_iter = std::max(1, sys->opt.max_iter);
  mtf_status status = MTF_OK;
  if (!mixed) {
    status = gmres_core(sys, nrhs, b_dev, x_dev, MV_FP64, sys->opt.tol, max_iter, iters, restarts, rel, s);
  } else {
    // FP64 iterative refinement: r = b - M x with FP64 accumulation over the
    // FP32-stored operator; each correction is one FGMRES cycle in FP32
    // (fgmres_cycle32) that adds its update to x.  A cycle that ends on the
    // restart length is a restart (the next one starts from the new FP64
    // residual); one that reaches its tolerance ends a refinement step.
    if (G.b.n != size_t(n) * nrhs * 2) G.b.alloc(size_t(n) * nrhs * 2);  // residual
    const size_t vec_bytes = size_t(n) * nrhs * 2 * sizeof(double);
    double* hN = G.h.p + 4 * size_t(m + 1) * nrhs;
    double* hostN = G.h_host + 4 * size_t(m + 1) * nrhs;
    std::vector<double> bnorm(nrhs);
    MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(b_dev, n, hN, G.w.p, n));
    MTF_CUDA(cudaMemcpyAsync(hostN, hN, size_t(nrhs) * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < nrhs; ++c) bnorm[c] = hostN[2 * c] > 0 ? hostN[2 * c] : 1.0;
    MTF_CUDA(cudaMemsetAsync(x_dev, 0, vec_bytes, s));
    const int max_ref = std::max(1, sys->opt.max_refine);
    int total = 0;
    // learned correction: used while it keeps the FP64 residual falling; a
    // cycle that fails to reduce it by 5% falls back to plain block-OSRC
    sys->learned_active = sys->opt.learned && sys->learned && sys->opt.precond == MTF_PRECOND_OSRC;
    double prev_rmax = -1.0;
    for (int it = 0;; ++it) {
      if (it == 0) {
        MTF_CUDA(cudaMemcpyAsync(G.b.p, b_dev, vec_bytes, cudaMemcpyDeviceToDevice, s));
      } else {
        // b - M x with the FP64 blocks (residual_fp64) or the FP32-stored ones
        launch_matvec_kind(sys, sys->opt.residual_fp64 ? MV_FP64 : MV_FP32_ACC64, x_dev, n, G.w.p, n, nrhs, s);
        MTF_LAUNCH(KID_SUB, s, k_sub<<<nblk(n * nrhs * 2, 256), 256, 0, s>>>(b_dev, G.w.p, G.b.p, n * nrhs * 2));
      }
      MTF_LAUNCH(KID_NORM, s, k_norm_scale<<<nrhs, 1024, 0, s>>>(G.b.p, n, hN, G.w.p, n));
      MTF_CUDA(cudaMemcpyAsync(hostN, hN, size_t(nrhs) * 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      MTF_CUDA(cudaStreamSynchronize(s));
      double rmax = 0;
      for (int c = 0; c < nrhs; ++c) {
        rel[c] = hostN[2 * c] / bnorm[c];
        if (!std::isfinite(rel[c])) status = MTF_ERR_NAN;
        rmax = std::max(rmax, rel[c]);
      }
      if (status != MTF_OK) break;
      if (rmax <= sys->opt.tol) break;
      if (sys->learned_active && prev_rmax > 0 && rmax > 0.95 * prev_rmax) sys->learned_active = false;
      prev_rmax = rmax;
      if (refinements >= max_ref || total >= max_iter) {
        status = MTF_ERR_NOCONV;
        break;
      }
      // right-hand sides already converged get a zero residual
      for (int c = 0; c < nrhs; ++c)
        if (rel[c] <= sys->opt.tol)
          MTF_CUDA(cudaMemsetAsync(G.b.p + 2 * size_t(c) * n, 0, size_t(n) * 2 * sizeof(double), s));
      const double tol_min = sys->opt.inner_tol_min > 0 ? sys->opt.inner_tol_min : 1e-5;
      const double inner_tol = std::min(0.5, std::max(tol_min, 0.3 * sys->opt.tol / rmax));
      std::vector<int> it_in(nrhs, 0);
      bool reached = false;
      // 4 or more right-hand sides share one block space (with or without
      // the learned correction, which both cycles apply after block-OSRC)
      if (sys->opt.block_krylov && nrhs >= kBlockMinRhs)
        status = fgmres_block32(sys, nrhs, G.b.p, x_dev, inner_tol, max_iter - total, it_in, reached, s);
      else
        status = fgmres_cycle32(sys, nrhs, G.b.p, x_dev, inner_tol, max_iter - total, it_in, reached, s, it);
      if (status != MTF_OK) break;
      int mx = 0;
      for (int c = 0; c < nrhs; ++c) {
        iters[c] += it_in[c];
        mx = std::max(mx, it_in[c]);
      }
      total += mx;
      ++restarts;
      if (reached) ++refinements;
    }
    MTF_CUDA(cudaStreamSynchronize(s));
  }
  if (st) {
    st->iterations = *std::max_element(iters.begin(), iters.end());
    st->restarts = restarts;
    st->refinements = refinements;
    st->converged = status == MTF_OK;
    st->rel_residual = *std::max_element(rel.begin(), rel.end());
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st->launch_seconds = sys->t_launch;
    st->lsq_seconds = sys->t_lsq;
    st->wait_seconds = sys->t_wait;
  }
  return status;
}

}  // namespace mtf
