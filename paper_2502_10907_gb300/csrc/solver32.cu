// FP32-basis inner FGMRES of the mixed-precision solve.  The outer loop
// (solve()) forms the true residual r = b - M x with FP64 accumulation; one
// call here runs one flexible GMRES cycle on M d = r from d = 0 and adds
// x += Z y.  Everything the cycle streams is FP32: the Krylov basis V, the
// preconditioned directions Z = P V, the matvec input and output.  Inner
// products and norms are reduced in FP64 (per-lane FP32 partial sums over at
// most a few dozen terms, FP64 across lanes and CTAs), so the Hessenberg
// entries keep FP64 accuracy of the FP32 data.  The cycle only has to reach
// the inner tolerance (>= 1e-5 relative to ||r||); the FP64 residual of the
// next outer step corrects its rounding.
//
// Vectors are stored with a padded stride ldn (a multiple of 64 complex
// entries) so that every vector starts on a 512-byte boundary and the
// streaming kernels read two complex entries per lane as one float4; the
// padding is zero at allocation and every kernel keeps it zero.
#include <algorithm>
#include <cmath>

#include "common.h"
#include "krylov_host.h"

namespace mtf {

struct Gmres32Work {
  int nrhs = 0, m = 0;
  int64_t n = 0, ldn = 0;
  bool pre = false;
  DevBuf<float> V, Z, w;
  // h: kBatch slots, one per Arnoldi column j of a batch; slot layout (complex
  // entries, index i * nrhs + c): hA (j+1) x nrhs, hB (j+1) x nrhs, ||w|| nrhs,
  // then nrhs real sums of squares
  DevBuf<double> h, y;
  double* h_host = nullptr;
  ~Gmres32Work() {
    if (h_host) cudaFreeHost(h_host);
  }
};

void destroy_gmres32(Gmres32Work* w) { delete w; }

static inline unsigned nb(int64_t n, int t) { return unsigned((n + t - 1) / t); }

// h[i*hst + c] += sum_{k in segment} conj(V_i^c[k]) w^c[k].  CTA = one
// segment of kDotSeg entries of w (staged in shared memory as float4 pairs)
// x 32 basis vectors (4 per warp); every lane keeps all 16 of its float4
// loads in flight at once.  Grid (segments, ceil(rows/32), c); V_i^c starts at
// V + 2 (c ldv + i ldn).
constexpr int kDotSeg = 256;

__global__ void __launch_bounds__(256) k_dots32(const float* __restrict__ V, const float* __restrict__ w, int64_t ldn,
                                                int64_t ldv, int rows, double* __restrict__ h, int hst) {
  __shared__ float4 ws4[kDotSeg / 2];
  constexpr int RW = 4, NQ = kDotSeg / 64;  // float4 per lane
  const int c = blockIdx.z;
  const int64_t k0 = int64_t(blockIdx.x) * kDotSeg;
  const int nq = int(min(ldn - k0, int64_t(kDotSeg)) >> 1);
  const float4* wc = reinterpret_cast<const float4*>(w + 2 * (int64_t(c) * ldn + k0));
  if (threadIdx.x < nq) ws4[threadIdx.x] = wc[threadIdx.x];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * (8 * RW) + warp * RW;
  if (i0 >= rows) return;
  const float4* v[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r)
    v[r] = reinterpret_cast<const float4*>(V + 2 * (int64_t(c) * ldv + int64_t(min(i0 + r, rows - 1)) * ldn + k0));
  float4 a[NQ][RW];
#pragma unroll
  for (int u = 0; u < NQ; ++u)
#pragma unroll
    for (int r = 0; r < RW; ++r)
      a[u][r] = lane + 32 * u < nq ? v[r][lane + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
  float ar[RW], ai[RW];
#pragma unroll
  for (int r = 0; r < RW; ++r) ar[r] = ai[r] = 0.f;
#pragma unroll
  for (int u = 0; u < NQ; ++u) {
    const float4 x = lane + 32 * u < nq ? ws4[lane + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      ar[r] += a[u][r].x * x.x + a[u][r].y * x.y + a[u][r].z * x.z + a[u][r].w * x.w;
      ai[r] += a[u][r].x * x.y - a[u][r].y * x.x + a[u][r].z * x.w - a[u][r].w * x.z;
    }
  }
  // FP32 warp sums (32 lane partials), FP64 accumulation over segments
#pragma unroll
  for (int r = 0; r < RW; ++r) {
    float sr = ar[r], si = ai[r];
#pragma unroll
    for (int s2 = 16; s2 > 0; s2 >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, s2);
      si += __shfl_xor_sync(0xffffffffu, si, s2);
    }
    if (lane == 0 && i0 + r < rows) {
      atomicAdd(h + 2 * (int64_t(i0 + r) * hst + c), double(sr));
      atomicAdd(h + 2 * (int64_t(i0 + r) * hst + c) + 1, double(si));
    }
  }
}

// w^c -= sum_{i<j} V_i^c h_i^c (h_i^c at h[i*hst + c], FP64, used as FP32); optionally
// ss[c] += ||w^c||^2 after the update.  CTA = 64 consecutive entries (a float4
// pair per lane) x 8 groups of basis vectors (i = grp mod 8), the group sums
// combined in shared memory; grid (ldn / 64, c).
__global__ void __launch_bounds__(256) k_axpy32(const float* __restrict__ V, const double* __restrict__ h, int j,
                                                int64_t ldn, int64_t ldv, int hst, float* __restrict__ w,
                                                double* __restrict__ ss) {
  const int c = blockIdx.y;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t q = int64_t(blockIdx.x) * 32 + lane;  // float4 index within a vector
  __shared__ float4 part[8][32];
  extern __shared__ float2 hs[];
  const double2* hc = reinterpret_cast<const double2*>(h) + c;
  for (int t = threadIdx.x; t < j; t += blockDim.x) {
    const double2 hv = hc[int64_t(t) * hst];
    hs[t] = make_float2(float(hv.x), float(hv.y));
  }
  __syncthreads();
  const int64_t ldq = ldn >> 1;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (q < ldq) {
    const float4* v = reinterpret_cast<const float4*>(V + 2 * int64_t(c) * ldv) + q;
#pragma unroll 16
    for (int i = grp; i < j; i += 8) {
      const float4 a = v[int64_t(i) * ldq];
      const float2 hv = hs[i];
      acc.x += a.x * hv.x - a.y * hv.y;
      acc.y += a.x * hv.y + a.y * hv.x;
      acc.z += a.z * hv.x - a.w * hv.y;
      acc.w += a.z * hv.y + a.w * hv.x;
    }
  }
  part[grp][lane] = acc;
  __syncthreads();
  if (grp != 0) return;
  float sq = 0.f;
  if (q < ldq) {
    float4 t = part[0][lane];
#pragma unroll
    for (int g = 1; g < 8; ++g) {
      const float4 p = part[g][lane];
      t.x += p.x;
      t.y += p.y;
      t.z += p.z;
      t.w += p.w;
    }
    float4* x = reinterpret_cast<float4*>(w + 2 * int64_t(c) * ldn) + q;
    float4 o = *x;
    o.x -= t.x;
    o.y -= t.y;
    o.z -= t.z;
    o.w -= t.w;
    *x = o;
    sq = o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
  }
  if (ss) {
    for (int s2 = 16; s2 > 0; s2 >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s2);
    if (lane == 0) atomicAdd(ss + c, double(sq));
  }
}

// out^c = w^c / sqrt(ss[c]) over the padded length (zero if ss is 0);
// nrm[c] = (sqrt(ss[c]), 0).  grid (ldn / 512, c), one float4 per thread.
__global__ void __launch_bounds__(256) k_scale32(const float* __restrict__ w, int64_t ldn, const double* __restrict__ ss,
                                                 double* __restrict__ nrm, float* __restrict__ out, int64_t ldo) {
  const int c = blockIdx.y;
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  __shared__ float sinv;  // one FP64 square root per CTA, not per thread
  if (threadIdx.x == 0) {
    const double t = sqrt(ss[c]);
    sinv = t > 0 ? float(1.0 / t) : 0.f;
    if (blockIdx.x == 0) {
      nrm[2 * c] = t;
      nrm[2 * c + 1] = 0.0;
    }
  }
  __syncthreads();
  if (q >= (ldn >> 1)) return;
  const float inv = sinv;
  float4 a = reinterpret_cast<const float4*>(w + 2 * int64_t(c) * ldn)[q];
  a.x *= inv;
  a.y *= inv;
  a.z *= inv;
  a.w *= inv;
  reinterpret_cast<float4*>(out + 2 * int64_t(c) * ldo)[q] = a;
}

// ss[c] += ||r^c||^2 of an FP64 vector (column stride n)
__global__ void __launch_bounds__(256) k_sqnorm64(const double* __restrict__ r, int64_t n, double* __restrict__ ss) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double sq = 0;
  if (k < n) {
    const double2 a = reinterpret_cast<const double2*>(r)[int64_t(c) * n + k];
    sq = a.x * a.x + a.y * a.y;
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, s2);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) t += red[q];
    atomicAdd(ss + c, t);
  }
}

// V_0^c = r^c / sqrt(ss[c]) in FP32 (rows < n; the padding stays zero)
__global__ void __launch_bounds__(256) k_start32(const double* __restrict__ r, int64_t n, const double* __restrict__ ss,
                                                 float* __restrict__ V, int64_t ldv) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double t = sqrt(ss[c]);
  const double inv = t > 0 ? 1.0 / t : 0.0;
  const double2 a = reinterpret_cast<const double2*>(r)[int64_t(c) * n + k];
  reinterpret_cast<float2*>(V + 2 * int64_t(c) * ldv)[k] = make_float2(float(a.x * inv), float(a.y * inv));
}

// x^c += sum_{i<j} Z_i^c y_i^c: FP32 basis, FP64 coefficients and FP64
// accumulation of the group sums into the FP64 iterate (column stride n).
// Same CTA shape as k_axpy32.
__global__ void __launch_bounds__(256) k_xupdate32(const float* __restrict__ Z, const double* __restrict__ y, int j,
                                                   int64_t ldn, int64_t ldz, int ldy, int64_t n,
                                                   double* __restrict__ x) {
  const int c = blockIdx.y;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t q = int64_t(blockIdx.x) * 32 + lane;
  __shared__ double2 part[8][2][32];
  extern __shared__ double2 ys[];
  const double2* yc = reinterpret_cast<const double2*>(y) + int64_t(c) * ldy;
  for (int t = threadIdx.x; t < j; t += blockDim.x) ys[t] = yc[t];
  __syncthreads();
  const int64_t ldq = ldn >> 1;
  double2 a0 = make_double2(0, 0), a1 = make_double2(0, 0);
  if (q < ldq) {
    const float4* v = reinterpret_cast<const float4*>(Z + 2 * int64_t(c) * ldz) + q;
#pragma unroll 4
    for (int i = grp; i < j; i += 8) {
      const float4 a = v[int64_t(i) * ldq];
      const double2 yv = ys[i];
      a0.x += double(a.x) * yv.x - double(a.y) * yv.y;
      a0.y += double(a.x) * yv.y + double(a.y) * yv.x;
      a1.x += double(a.z) * yv.x - double(a.w) * yv.y;
      a1.y += double(a.z) * yv.y + double(a.w) * yv.x;
    }
  }
  part[grp][0][lane] = a0;
  part[grp][1][lane] = a1;
  __syncthreads();
  if (grp != 0 || q >= ldq) return;
  double2 t0 = make_double2(0, 0), t1 = make_double2(0, 0);
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    t0.x += part[g][0][lane].x;
    t0.y += part[g][0][lane].y;
    t1.x += part[g][1][lane].x;
    t1.y += part[g][1][lane].y;
  }
  double2* xc = reinterpret_cast<double2*>(x) + int64_t(c) * n;
  const int64_t k = 2 * q;
  if (k < n) {
    double2 o = xc[k];
    o.x += t0.x;
    o.y += t0.y;
    xc[k] = o;
  }
  if (k + 1 < n) {
    double2 o = xc[k + 1];
    o.x += t1.x;
    o.y += t1.y;
    xc[k + 1] = o;
  }
}

static void launch_dots32(const float* V, const float* w, int64_t ldn, int64_t ldv, int rows, double* h, int nrhs,
                          cudaStream_t s) {
  dim3 g{nb(ldn, kDotSeg), nb(rows, 32), unsigned(nrhs)};
  MTF_LAUNCH(KID_DOTS, s, k_dots32<<<g, 256, 0, s>>>(V, w, ldn, ldv, rows, h, nrhs));
}

// Arnoldi columns enqueued back to back before the host reads their
// Hessenberg entries: CGS2 needs no host result, only the stopping test does,
// so at most kBatch - 1 iterations per cycle are computed beyond the one that
// meets the tolerance (they are discarded) while kBatch - 1 of every kBatch
// host round trips disappear.
constexpr int kBatch = 8;

// doubles of the Hessenberg slot of column j
static inline size_t slot_len(int j, int nrhs) { return size_t(4 * (j + 1) + 4) * nrhs; }

mtf_status fgmres_cycle32(mtf_system sys, int nrhs, const double* r_dev, double* x_dev, double tol, int max_iter,
                          std::vector<int>& iters, bool& reached, cudaStream_t s) {
  mtf_mesh msh = sys->mesh;
  const int64_t n = msh->n_total;
  const int64_t ldn = (n + 63) & ~int64_t(63);
  const int m = std::max(1, sys->opt.restart);
  const bool pre = sys->opt.precond == MTF_PRECOND_OSRC;
  if (!sys->gw32) sys->gw32 = new Gmres32Work();
  Gmres32Work& G = *sys->gw32;
  if (G.nrhs != nrhs || G.m != m || G.n != n || G.pre != pre) {
    G.V.alloc(size_t(m + 1) * ldn * nrhs * 2);
    MTF_CUDA(cudaMemsetAsync(G.V.p, 0, G.V.n * sizeof(float), s));
    if (pre) {
      G.Z.alloc(size_t(m) * ldn * nrhs * 2);
      MTF_CUDA(cudaMemsetAsync(G.Z.p, 0, G.Z.n * sizeof(float), s));
    } else {
      G.Z.release();
    }
    G.w.alloc(size_t(ldn) * nrhs * 2);
    MTF_CUDA(cudaMemsetAsync(G.w.p, 0, G.w.n * sizeof(float), s));
    G.h.alloc(size_t(kBatch) * slot_len(m - 1, nrhs));
    G.y.alloc(size_t(m + 1) * nrhs * 2);
    if (G.h_host) cudaFreeHost(G.h_host);
    G.h_host = nullptr;
    MTF_CUDA(cudaMallocHost(&G.h_host, G.h.n * sizeof(double)));
    G.nrhs = nrhs;
    G.m = m;
    G.n = n;
    G.ldn = ldn;
    G.pre = pre;
  }
  const int ldh = m + 1;
  const int64_t ldv = int64_t(m + 1) * ldn, ldz = int64_t(m) * ldn;
  const size_t slot = slot_len(m - 1, nrhs);

  // V_0 = r / ||r|| (sums of squares in slot 0)
  MTF_CUDA(cudaMemsetAsync(G.h.p, 0, size_t(nrhs) * sizeof(double), s));
  MTF_LAUNCH(KID_NORM, s, k_sqnorm64<<<dim3(nb(n, 256), unsigned(nrhs)), 256, 0, s>>>(r_dev, n, G.h.p));
  MTF_LAUNCH(KID_NORM, s, k_start32<<<dim3(nb(n, 256), unsigned(nrhs)), 256, 0, s>>>(r_dev, n, G.h.p, G.V.p, ldv));
  MTF_CUDA(cudaMemcpyAsync(G.h_host, G.h.p, size_t(nrhs) * sizeof(double), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  HostArnoldi ha(m, nrhs);
  std::vector<int> active(nrhs);
  bool any = false;
  for (int c = 0; c < nrhs; ++c) {
    const double rn = std::sqrt(G.h_host[c]);
    if (!std::isfinite(rn)) return MTF_ERR_NAN;
    ha.start(c, rn);
    active[c] = rn > 0;
    any = any || active[c];
  }
  reached = !any;
  if (!any) return MTF_OK;

  mtf_status status = MTF_OK;
  const size_t hsm = size_t(m + 1) * sizeof(float2);
  const size_t ysm = size_t(m + 1) * sizeof(double2);
  if (hsm > 48 * 1024 || ysm > 40 * 1024) {
    MTF_REQUIRE(ysm <= 200 * 1024, MTF_ERR_ARG, "restart length too large for the FP32 inner solver");
    MTF_CUDA(cudaFuncSetAttribute(k_axpy32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hsm)));
    MTF_CUDA(cudaFuncSetAttribute(k_xupdate32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ysm)));
  }
  const dim3 ga{nb(ldn / 2, 32), unsigned(nrhs)};
  const dim3 gs{nb(ldn / 2, 256), unsigned(nrhs)};
  const int jend = std::min(m, std::max(1, max_iter));
  std::vector<double> hcol;
  bool stop = false;
  for (int j0 = 0; j0 < jend && !stop; j0 += kBatch) {
    const int nbat = std::min(kBatch, jend - j0);
    // the batch's Hessenberg slots are cleared once and copied back once
    MTF_CUDA(cudaMemsetAsync(G.h.p, 0, size_t(nbat) * slot * sizeof(double), s));
    for (int b = 0; b < nbat; ++b) {
      const int j = j0 + b;
      const float* vj = G.V.p + 2 * size_t(j) * ldn;
      if (pre) {
        float* zj = G.Z.p + 2 * size_t(j) * ldn;
        launch_osrc_apply_f32(sys, vj, ldv, zj, ldz, nrhs, s);
        launch_matvec_f32(sys, zj, ldz, G.w.p, ldn, nrhs, s);
      } else {
        launch_matvec_f32(sys, vj, ldv, G.w.p, ldn, nrhs, s);
      }
      // CGS2 with FP64 accumulation of the FP32 partial sums
      double* hA = G.h.p + size_t(b) * slot;
      double* hB = hA + 2 * size_t(j + 1) * nrhs;
      double* hN = hB + 2 * size_t(j + 1) * nrhs;
      double* ss = hN + 2 * nrhs;
      launch_dots32(G.V.p, G.w.p, ldn, ldv, j + 1, hA, nrhs, s);
      MTF_LAUNCH(KID_AXPY, s, k_axpy32<<<ga, 256, hsm, s>>>(G.V.p, hA, j + 1, ldn, ldv, nrhs, G.w.p, nullptr));
      launch_dots32(G.V.p, G.w.p, ldn, ldv, j + 1, hB, nrhs, s);
      MTF_LAUNCH(KID_AXPY, s, k_axpy32<<<ga, 256, hsm, s>>>(G.V.p, hB, j + 1, ldn, ldv, nrhs, G.w.p, ss));
      MTF_LAUNCH(KID_NORM, s, k_scale32<<<gs, 256, 0, s>>>(G.w.p, ldn, ss, hN, G.V.p + 2 * size_t(j + 1) * ldn, ldv));
    }
    MTF_CUDA(cudaMemcpyAsync(G.h_host, G.h.p, (size_t(nbat - 1) * slot + slot_len(j0 + nbat - 1, nrhs)) * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < nbat && !stop; ++b) {
      const int j = j0 + b;
      const double* hostA = G.h_host + size_t(b) * slot;
      const double* hostB = hostA + 2 * size_t(j + 1) * nrhs;
      const double* hostN = hostB + 2 * size_t(j + 1) * nrhs;
      hcol.assign(2 * size_t(j + 1), 0.0);
      bool all_done = true;
      for (int c = 0; c < nrhs; ++c) {
        if (!active[c]) continue;
        for (int q = 0; q <= j; ++q) {
          hcol[2 * q] = hostA[2 * (size_t(q) * nrhs + c)] + hostB[2 * (size_t(q) * nrhs + c)];
          hcol[2 * q + 1] = hostA[2 * (size_t(q) * nrhs + c) + 1] + hostB[2 * (size_t(q) * nrhs + c) + 1];
        }
        const double hn = hostN[2 * c];
        const double est = ha.add_column(c, j, hcol.data(), hn);
        ++iters[c];
        if (!std::isfinite(est)) status = MTF_ERR_NAN;
        if (est <= tol || hn == 0.0) active[c] = 0;
        all_done = all_done && !active[c];
      }
      if (status != MTF_OK) {
        check_matvec_stream(sys, s);
        return status;
      }
      if (all_done) {
        reached = true;
        stop = true;
      }
    }
  }
  check_matvec_stream(sys, s);
  // x += Z y (flexible) or V y, y = R^{-1} g per right-hand side
  std::vector<double> yhost(size_t(m + 1) * nrhs * 2);
  const int jmax = ha.solve(yhost);
  for (double v : yhost)
    if (!std::isfinite(v)) return MTF_ERR_NAN;
  if (jmax > 0) {
    MTF_CUDA(cudaMemcpyAsync(G.y.p, yhost.data(), yhost.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    MTF_LAUNCH(KID_AXPY, s, k_xupdate32<<<ga, 256, size_t(jmax) * sizeof(double2), s>>>(
        pre ? G.Z.p : G.V.p, G.y.p, jmax, ldn, pre ? ldz : ldv, ldh, n, x_dev));
    MTF_CUDA(cudaStreamSynchronize(s));  // yhost is released on return
  }
  return status;
}

}  // namespace mtf
