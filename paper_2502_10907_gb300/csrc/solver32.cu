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
#include <atomic>
#include <cmath>


#include "bulk.h"
#include "common.h"
#include "krylov_host.h"

namespace mtf {

struct Gmres32Work {
  int nrhs = 0, m = 0;
  int64_t n = 0, ldn = 0;
  bool pre = false;
  DevBuf<float> V, Z, w;
  // recycled space of the previous cycle of the same solve: C = V Q in the
  // first rec_k columns of V; U = Z R^{-1} (M U = C) is kept as the first
  // rec_k columns of Z and the factor R (host, per rhs), and applied as
  // U c = Z (R^{-1} c)
  int rec_k = 0;
  DevBuf<float> RC, RQ;
  std::vector<std::vector<std::complex<double>>> rec_R;  // per rhs: R (rec_kc x rec_kc, column-major, ld rec_k)
  std::vector<int> rec_kc;
  // h: kBatch slots, one per Arnoldi column j of a batch; slot layout (complex
  // entries, index i * nrhs + c): t (j+1) x nrhs, s (j+1) x nrhs, coef 2 nrhs
  // (alpha, h_j), ||w|| nrhs, then nrhs real sums of squares
  DevBuf<double> h, y;
  double* h_host = nullptr;
  ~Gmres32Work() {
    if (h_host) cudaFreeHost(h_host);
  }
};

void destroy_gmres32(Gmres32Work* w) { delete w; }

static inline unsigned nb(int64_t n, int t) { return unsigned((n + t - 1) / t); }

// Fused reduction of the delayed CGS2 step (one pass over the basis):
//   t[i*hst + c] += sum_k conj(V_i^c[k]) w^c[k]   and
//   s[i*hst + c] += sum_k conj(V_i^c[k]) V_jq^c[k]   for i < rows,
// V_i^c starting at V + 2 (c ldv + i ldn).  The basis is staged in shared
// memory by the bulk-copy engine: a persistent CTA per SM takes units
// (right-hand side c, segment of kDtL entries, group of kDtR basis vectors)
// in turn.  A producer warp copies
// the unit's kDtR vector slices and the matching slices of w and q~ into a
// ring of kDtS stages (one "full" mbarrier per stage); kDtCons consumer warps,
// kDtRW vectors each, form the four partial sums per vector from shared
// memory, reduce them over the warp and add them into t and s (FP64), then
// release the stage ("empty" mbarrier).  The copies of the next units are in
// flight while a unit is reduced, so the basis streams at a steady rate
// instead of in one burst per CTA wave (measured on the split sphere: 14 %
// less time than one register-staged pass per CTA; 4 KB slices of 16
// vectors beat 2 KB slices and 16 warps of one vector).  Every wait is
// bounded (~0.5 s): on timeout the kernel sets *err and its warps leave.
#ifndef MTF_DT_L
#define MTF_DT_L 512
#endif
#ifndef MTF_DT_RW
#define MTF_DT_RW 2
#endif
#ifndef MTF_DT_CONS
#define MTF_DT_CONS 8
#endif
#ifndef MTF_DT_S
#define MTF_DT_S 3
#endif
constexpr int kDtL = MTF_DT_L;            // complex entries per slice (a multiple of 64)
constexpr int kDtRW = MTF_DT_RW;          // basis vectors per consumer warp
constexpr int kDtCons = MTF_DT_CONS;      // consumer warps
constexpr int kDtR = kDtRW * kDtCons;     // basis vectors per unit
constexpr int kDtSliceB = kDtL * 8;       // bytes of one slice
constexpr int kDtSB = (kDtR + 2) * kDtSliceB;
constexpr int kDtS = MTF_DT_S;
static_assert(kDtL % 64 == 0 && (kDtRW == 1 || kDtRW == 2 || kDtRW == 4), "unsupported dot-kernel tiling");
constexpr size_t kDtSmem = size_t(kDtS) * kDtSB + size_t(kDtS) * 2 * sizeof(uint64_t);
static_assert(kDtSmem <= 232448, "stage ring above the per-CTA shared-memory limit");
constexpr uint64_t kDtWaitNs = 500000000ull;

__global__ void __launch_bounds__((kDtCons + 1) * 32, 1)
    k_dots_tma(const float* __restrict__ V, const float* __restrict__ w, int64_t ldn, int64_t ldv, int rows, int jq,
               double* __restrict__ t, double* __restrict__ sq, int hst, int nrhs, unsigned* __restrict__ err) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(kDtS) * kDtSB);
  uint64_t* empty = full + kDtS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nseg = int((ldn + kDtL - 1) / kDtL), nrg = (rows + kDtR - 1) / kDtR;
  const int n_units = nseg * nrg * nrhs;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kDtS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], kDtCons);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (warp == kDtCons) {
    // producer: one lane issues every copy
    if (lane != 0) return;
    int k = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++k) {
      const int seg = u % nseg, rg = (u / nseg) % nrg, c = u / (nseg * nrg);
      const int st = k % kDtS;
      if (!mbar_wait_bounded(&empty[st], (uint32_t(k / kDtS) & 1u) ^ 1u, kDtWaitNs)) {
        atomicExch(err, 1u);
        return;
      }
      const int64_t k0 = int64_t(seg) * kDtL;
      const uint32_t bytes = uint32_t(min(int64_t(kDtL), ldn - k0)) * 8u;
      const int i0 = rg * kDtR, nr = min(kDtR, rows - i0);
      mbar_arrive_expect_tx(&full[st], uint32_t(nr + 2) * bytes);
      unsigned char* sb = smem + size_t(st) * kDtSB;
      const float* Vc = V + 2 * (int64_t(c) * ldv + k0);
      for (int r = 0; r < nr; ++r) bulk_g2s(sb + r * kDtSliceB, Vc + 2 * int64_t(i0 + r) * ldn, bytes, &full[st]);
      bulk_g2s(sb + kDtR * kDtSliceB, w + 2 * (int64_t(c) * ldn + k0), bytes, &full[st]);
      bulk_g2s(sb + (kDtR + 1) * kDtSliceB, Vc + 2 * int64_t(jq) * ldn, bytes, &full[st]);
    }
    return;
  }
  int k = 0;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++k) {
    const int st = k % kDtS;
    if (!mbar_wait_bounded(&full[st], uint32_t(k / kDtS) & 1u, kDtWaitNs)) {
      if (lane == 0) atomicExch(err, 1u);
      return;
    }
    const int seg = u % nseg, rg = (u / nseg) % nrg, c = u / (nseg * nrg);
    const int64_t k0 = int64_t(seg) * kDtL;
    const int nq = int(min(int64_t(kDtL), ldn - k0) >> 1);  // float4 (two complex) per slice
    const int i0 = rg * kDtR, nr = min(kDtR, rows - i0);
    const int r0 = kDtRW * warp;
    if (r0 < nr) {
      const unsigned char* sb = smem + size_t(st) * kDtSB;
      const float4* xw = reinterpret_cast<const float4*>(sb + kDtR * kDtSliceB);
      const float4* xq = reinterpret_cast<const float4*>(sb + (kDtR + 1) * kDtSliceB);
      const float4* a[kDtRW];
#pragma unroll
      for (int r = 0; r < kDtRW; ++r)
        a[r] = reinterpret_cast<const float4*>(sb + min(r0 + r, nr - 1) * kDtSliceB);  // repeats are discarded
      float v[4 * kDtRW];
#pragma unroll
      for (int q = 0; q < 4 * kDtRW; ++q) v[q] = 0.f;
#pragma unroll 4
      for (int e = lane; e < nq; e += 32) {
        const float4 x = xw[e], y = xq[e];
#pragma unroll
        for (int r = 0; r < kDtRW; ++r) {
          const float4 b = a[r][e];
          v[4 * r] += b.x * x.x + b.y * x.y + b.z * x.z + b.w * x.w;  // conj(V) w
          v[4 * r + 1] += b.x * x.y - b.y * x.x + b.z * x.w - b.w * x.z;
          v[4 * r + 2] += b.x * y.x + b.y * y.y + b.z * y.z + b.w * y.w;  // conj(V) q~
          v[4 * r + 3] += b.x * y.y - b.y * y.x + b.z * y.w - b.w * y.z;
        }
      }
      // lane (32 / (4 kDtRW)) q ends with the warp total of value q
      WarpTransposeSum<4 * kDtRW>::run(v, lane, 16);
      constexpr int SH = kDtRW == 1 ? 3 : (kDtRW == 2 ? 2 : 1);
      if ((lane & ((1 << SH) - 1)) == 0) {
        const int q = lane >> SH, r = q >> 2, kind = q & 3;
        if (r0 + r < nr)
          atomicAdd((kind < 2 ? t : sq) + 2 * (int64_t(i0 + r0 + r) * hst + c) + (kind & 1), double(v[0]));
      }
    }
    // release the stage: order this warp's shared reads before the next bulk write
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
}

// Coefficients of the delayed CGS2 step for column j (j > 0) from
// s_i = <V_i, q~_j> (i < j), sigma = <q~_j, q~_j> and t_i = <V_i, w>:
//   alpha = sqrt(sigma - sum |s_i|^2)   (norm of q~_j - sum V_i s_i),
//   h_j   = (t_j - sum conj(s_i) t_i) / alpha   (= <q_j, w>);
// for j = 0 the start vector is final: alpha = 1, h_0 = t_0.  A vanishing
// q~_j (a right-hand side with zero residual, or an exhausted Krylov space)
// keeps alpha = 1: nothing is divided by zero and the subdiagonal beta alpha
// reports the breakdown through beta.
template <class R>
__device__ __forceinline__ void dcgs_coef(R sigma, R s2, R pr, R pi, R tjr, R tji, bool first, R& alpha, R& hr,
                                          R& hi) {
  alpha = R(1);
  const R d = sigma - s2;
  if (!first && sigma > R(0) && d > R(1e-12) * sigma) alpha = sqrt(d);
  hr = (tjr - pr) / alpha;
  hi = (tji - pi) / alpha;
}

// Update of the delayed CGS2 step, one pass over V_0 .. V_{j-1}:
//   q_j = (q~_j - sum_{i<j} V_i s_i) / alpha        (written over V_j = q~_j)
//   w  <- w - sum_{i<j} V_i t_i - h_j q_j            (in place)
// and ss[c] += ||w||^2 after the update.  t, s at [i*hst + c] (FP64, used as
// FP32).  Every CTA forms alpha and h_j itself in FP32 from the staged t, s;
// CTA 0 of each right-hand side also forms them in FP64 and stores
// coef[c] = (alpha, 0), coef[nrhs + c] = h_j for the Hessenberg matrix.
// CTA = 64 consecutive entries (a float4 pair per lane) x 8 groups of basis
// vectors (i = grp mod 8), the group sums combined in shared memory; grid
// (ldn / 64, c).
__global__ void __launch_bounds__(256) k_axpy2_32(float* __restrict__ V, const double* __restrict__ t,
                                                  const double* __restrict__ sq, double* __restrict__ coef,
                                                  int j, int j0, int nrhs, int64_t ldn, int64_t ldv,
                                                  float* __restrict__ w, double* __restrict__ ss) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int c = blockIdx.y;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t q = int64_t(blockIdx.x) * 32 + lane;  // float4 index within a vector
  __shared__ float4 part_t[8][32], part_s[8][32];
  __shared__ float red[3][8];
  __shared__ double redd[3][8];
  __shared__ float cf[3];
  extern __shared__ float2 hs[];  // t_i at hs[i], s_i at hs[j + i]
  const bool lead = blockIdx.x == 0;
  // the first 8 basis columns of this group are loaded before the
  // coefficients are formed, so that their latency overlaps the prologue
  const int64_t ldq = ldn >> 1;
  float4* vb = reinterpret_cast<float4*>(V + 2 * int64_t(c) * ldv) + q;
  float4 pre[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int i = grp + 8 * u;
    pre[u] = (q < ldq && i < j) ? vb[int64_t(i) * ldq] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float s2 = 0.f, pr = 0.f, pi = 0.f;
  double s2d = 0, prd = 0, pid = 0;
  for (int u = threadIdx.x; u < j; u += blockDim.x) {
    const int64_t o = 2 * (int64_t(u) * nrhs + c);
    const double tr = t[o], ti = t[o + 1], sr = sq[o], si = sq[o + 1];
    const float2 tv = make_float2(float(tr), float(ti)), sv = make_float2(float(sr), float(si));
    hs[u] = tv;
    hs[j + u] = sv;
    s2 += sv.x * sv.x + sv.y * sv.y;
    pr += sv.x * tv.x + sv.y * tv.y;  // conj(s) t
    pi += sv.x * tv.y - sv.y * tv.x;
    if (lead) {
      s2d += sr * sr + si * si;
      prd += sr * tr + si * ti;
      pid += sr * ti - si * tr;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    pr += __shfl_xor_sync(0xffffffffu, pr, o);
    pi += __shfl_xor_sync(0xffffffffu, pi, o);
  }
  if (lane == 0) {
    red[0][grp] = s2;
    red[1][grp] = pr;
    red[2][grp] = pi;
  }
  if (lead) {
    for (int o = 16; o > 0; o >>= 1) {
      s2d += __shfl_xor_sync(0xffffffffu, s2d, o);
      prd += __shfl_xor_sync(0xffffffffu, prd, o);
      pid += __shfl_xor_sync(0xffffffffu, pid, o);
    }
    if (lane == 0) {
      redd[0][grp] = s2d;
      redd[1][grp] = prd;
      redd[2][grp] = pid;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, e = 0.f;
    for (int g = 0; g < 8; ++g) {
      a += red[0][g];
      b += red[1][g];
      e += red[2][g];
    }
    const int64_t oj = 2 * (int64_t(j) * nrhs + c);
    float alpha, hr, hi;
    dcgs_coef<float>(float(sq[oj]), a, b, e, float(t[oj]), float(t[oj + 1]), j == j0, alpha, hr, hi);
    cf[0] = 1.f / alpha;
    cf[1] = hr;
    cf[2] = hi;
    if (lead) {
      double ad = 0, bd = 0, ed = 0;
      for (int g = 0; g < 8; ++g) {
        ad += redd[0][g];
        bd += redd[1][g];
        ed += redd[2][g];
      }
      double alphad, hrd, hid;
      dcgs_coef<double>(sq[oj], ad, bd, ed, t[oj], t[oj + 1], j == j0, alphad, hrd, hid);
      coef[2 * c] = alphad;
      coef[2 * c + 1] = 0.0;
      coef[2 * (nrhs + c)] = hrd;
      coef[2 * (nrhs + c) + 1] = hid;
    }
  }
  __syncthreads();
  float4 at = make_float4(0.f, 0.f, 0.f, 0.f), as = at;
  if (q < ldq) {
    auto acc = [&](const float4 a, int i) {
      const float2 hv = hs[i], sv = hs[j + i];
      at.x += a.x * hv.x - a.y * hv.y;
      at.y += a.x * hv.y + a.y * hv.x;
      at.z += a.z * hv.x - a.w * hv.y;
      at.w += a.z * hv.y + a.w * hv.x;
      as.x += a.x * sv.x - a.y * sv.y;
      as.y += a.x * sv.y + a.y * sv.x;
      as.z += a.z * sv.x - a.w * sv.y;
      as.w += a.z * sv.y + a.w * sv.x;
    };
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (grp + 8 * u < j) acc(pre[u], grp + 8 * u);
#pragma unroll 16
    for (int i = grp + 64; i < j; i += 8) acc(vb[int64_t(i) * ldq], i);
  }
  part_t[grp][lane] = at;
  part_s[grp][lane] = as;
  __syncthreads();
  if (grp != 0) return;
  float sqn = 0.f;
  if (q < ldq) {
    float4 st = part_t[0][lane], ssum = part_s[0][lane];
#pragma unroll
    for (int g = 1; g < 8; ++g) {
      const float4 p1 = part_t[g][lane], p2 = part_s[g][lane];
      st.x += p1.x;
      st.y += p1.y;
      st.z += p1.z;
      st.w += p1.w;
      ssum.x += p2.x;
      ssum.y += p2.y;
      ssum.z += p2.z;
      ssum.w += p2.w;
    }
    const float ia = cf[0], hr = cf[1], hi = cf[2];
    float4* qv = vb + int64_t(j) * ldq;
    float4 qj = *qv;
    qj.x = (qj.x - ssum.x) * ia;
    qj.y = (qj.y - ssum.y) * ia;
    qj.z = (qj.z - ssum.z) * ia;
    qj.w = (qj.w - ssum.w) * ia;
    *qv = qj;
    float4* x = reinterpret_cast<float4*>(w + 2 * int64_t(c) * ldn) + q;
    float4 o = *x;
    o.x -= st.x + (hr * qj.x - hi * qj.y);
    o.y -= st.y + (hr * qj.y + hi * qj.x);
    o.z -= st.z + (hr * qj.z - hi * qj.w);
    o.w -= st.w + (hr * qj.w + hi * qj.z);
    *x = o;
    sqn = o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) sqn += __shfl_xor_sync(0xffffffffu, sqn, s2);
  if (lane == 0) atomicAdd(ss + c, double(sqn));
}

// w^c -= sum_{i<k} V_i^c t_i (t FP64 at [i * nrhs + c], interleaved
// complex) and ss[c] += ||w^c||^2 after the update: one classical
// Gram-Schmidt projection against k basis columns.  CTA = 64 entries x 8
// groups of columns (i = grp mod 8), grid (ldn / 64, c).
__global__ void __launch_bounds__(256) k_proj32(const float* __restrict__ V, const double* __restrict__ t, int k,
                                                int nrhs, int64_t ldn, int64_t ldv, float* __restrict__ w,
                                                double* __restrict__ ss) {
  const int c = blockIdx.y;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t q = int64_t(blockIdx.x) * 32 + lane;
  const int64_t ldq = ldn >> 1;
  __shared__ float4 part[8][32];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (q < ldq) {
    const float4* vb = reinterpret_cast<const float4*>(V + 2 * int64_t(c) * ldv) + q;
#pragma unroll 8
    for (int i = grp; i < k; i += 8) {
      const float4 a = vb[int64_t(i) * ldq];
      const int64_t o = 2 * (int64_t(i) * nrhs + c);
      const float hr = float(t[o]), hi = float(t[o + 1]);
      acc.x += a.x * hr - a.y * hi;
      acc.y += a.x * hi + a.y * hr;
      acc.z += a.z * hr - a.w * hi;
      acc.w += a.z * hi + a.w * hr;
    }
  }
  part[grp][lane] = acc;
  __syncthreads();
  if (grp != 0) return;
  float sqn = 0.f;
  if (q < ldq) {
    float4 st = part[0][lane];
#pragma unroll
    for (int g = 1; g < 8; ++g) {
      st.x += part[g][lane].x;
      st.y += part[g][lane].y;
      st.z += part[g][lane].z;
      st.w += part[g][lane].w;
    }
    float4* x = reinterpret_cast<float4*>(w + 2 * int64_t(c) * ldn) + q;
    float4 o = *x;
    o.x -= st.x;
    o.y -= st.y;
    o.z -= st.z;
    o.w -= st.w;
    *x = o;
    sqn = o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) sqn += __shfl_xor_sync(0xffffffffu, sqn, s2);
  if (lane == 0) atomicAdd(ss + c, double(sqn));
}

// out^c = w^c / sqrt(ss[c]) over the padded length (zero if ss is 0);
// nrm[c] = (sqrt(ss[c]), 0).  grid (ldn / 512, c), one float4 per thread.
__global__ void __launch_bounds__(256) k_scale32(const float* __restrict__ w, int64_t ldn, const double* __restrict__ ss,
                                                 double* __restrict__ nrm, float* __restrict__ out, int64_t ldo) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
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

// x^c += sum_{i<jc[c]} Z_i^c y_i^c: FP32 basis, FP64 coefficients and FP64
// accumulation of the group sums into the FP64 iterate (column stride n).
// Same CTA shape as k_axpy2_32.
__global__ void __launch_bounds__(256) k_xupdate32(const float* __restrict__ Z, const double* __restrict__ y,
                                                   const int* __restrict__ jc, int64_t ldn, int64_t ldz, int ldy,
                                                   int64_t n, double* __restrict__ x) {
  const int c = blockIdx.y;
  const int j = jc[c];  // columns of this right-hand side (others may hold anything)
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

static void launch_dots2_32(mtf_system sys, const float* V, const float* w, int64_t ldn, int64_t ldv, int rows,
                            int jq, double* t, double* sq, int nrhs, cudaStream_t s) {
  MTF_REQUIRE(ldn % 64 == 0 && ldv % 2 == 0 && (reinterpret_cast<uintptr_t>(V) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(w) & 15) == 0,
              MTF_ERR_ARG, "Krylov vectors must be 16-byte aligned with a stride of 64 entries");
  const int64_t units = ((ldn + kDtL - 1) / kDtL) * ((rows + kDtR - 1) / kDtR) * nrhs;
  if (units <= 0) return;
  stream_prepare(sys, s);
  // the shared-memory opt-in is set once per device, not on every launch
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load(std::memory_order_relaxed) & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_dots_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kDtSmem)));
    opted.fetch_or(bit);
  }
  const unsigned grid = unsigned(std::min<int64_t>(units, sys->mv_grid));
  MTF_LAUNCH(KID_DOTS, s,
             launch_pdl(k_dots_tma, dim3(grid), dim3((kDtCons + 1) * 32), kDtSmem, s, V, w, ldn, ldv, rows, jq, t, sq,
                        nrhs, nrhs, sys->d_mv_ctl.p + 2));
}

// Arnoldi columns enqueued back to back before the host reads their
// Hessenberg entries: the orthogonalisation needs no host result, only the
// stopping test does, so at most kBatch iterations per cycle are computed
// beyond the one that meets the tolerance (they are discarded) while
// kBatch - 1 of every kBatch host round trips disappear.
//
// Orthogonalisation: CGS2 with delayed re-orthogonalisation (the DCGS2
// variant of low-synchronisation Gram-Schmidt; Swirydowicz, Langou,
// Ananthan, Yang and Thomas, 2020).  Step j receives q~_j = V_j, once
// orthogonalised against q_0 .. q_{j-1}, applies the operator to it
// (z_j = P q~_j, w = M z_j), and in one pass over the basis both finishes
// q~_j (its second projection, q_j = (q~_j - sum V_i s_i) / alpha) and
// projects w once against q_0 .. q_j; the result w / ||w|| is q~_{j+1}.  Two
// passes over the basis per iteration instead of CGS2's four.  Finishing
// q~_j changes the previous Hessenberg column: with beta = ||w_{j-1}||,
// H[i, j-1] += beta s_i (i < j) and H[j, j-1] = beta alpha, so column j - 1 is
// final once step j's reduction is known and the host applies its Givens
// rotation then; the last column of a cycle keeps its once-projected
// values.  Since w was computed from q~_j, the solution update uses the
// vectors actually multiplied (z_j; without a preconditioner a copy of q~_j).
constexpr int kBatch = 8;

// doubles of the Hessenberg slot of column j
static inline size_t slot_len(int j, int nrhs) { return size_t(4 * (j + 1) + 8) * nrhs; }


// Out[:, j] = sum_{k < K} In[:, k] M[k, j] for j < ncol over n rows: In and Out
// complex FP32 columns of stride ldi / ldo, M complex FP32 column-major with
// leading dimension ldm.  CTA tile 128 rows x 32 columns, K in chunks of 32
// staged in shared memory; thread (row group, column group) holds 4 x 4
// complex sums.  (The recycling products C = V Q and U = Z R^-1.)
__global__ void __launch_bounds__(256) k_cgemm_nn(const float* __restrict__ In, int64_t ldi, const float* __restrict__ M,
                                                  int ldm, int K, int ncol, int64_t n, float* __restrict__ Out,
                                                  int64_t ldo) {
  __shared__ float2 a[32][128 + 1];  // a[k][row]
  __shared__ float2 b[32][32 + 1];   // b[k][col]
  const int tr = threadIdx.x & 31, tc = threadIdx.x >> 5;  // rows tr + 32 i, columns tc + 8 j
  const int64_t r0 = int64_t(blockIdx.x) * 128;
  const int c0 = blockIdx.y * 32;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 128; t += 256) {
      const int kk = t / 128, rr = t % 128;
      const int64_t row = r0 + rr;
      a[kk][rr] = (k0 + kk < K && row < n) ? reinterpret_cast<const float2*>(In + 2 * int64_t(k0 + kk) * ldi)[row]
                                           : make_float2(0.f, 0.f);
    }
    for (int t = threadIdx.x; t < 32 * 32; t += 256) {
      const int kk = t / 32, cc = t % 32;
      b[kk][cc] = (k0 + kk < K && c0 + cc < ncol)
                      ? reinterpret_cast<const float2*>(M)[int64_t(c0 + cc) * ldm + k0 + kk]
                      : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      float2 x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = a[kk][tr + 32 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) y[j] = b[kk][tc + 8 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(x[i].x, y[j].x, fmaf(-x[i].y, y[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(x[i].x, y[j].y, fmaf(x[i].y, y[j].x, acc[i][j].y));
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = r0 + tr + 32 * i;
    if (row >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = c0 + tc + 8 * j;
      if (col < ncol) reinterpret_cast<float2*>(Out + 2 * int64_t(col) * ldo)[row] = acc[i][j];
    }
  }
}

// Build the recycled space of a finished cycle for the next cycle of the same
// solve: per rhs c with k_c finished columns, H_c = Q_c R_c (host Givens
// data), C_c = V_c Q_c (orthonormal) in the first k_c columns of V, with
// M U_c = C_c for U_c = Z_c R_c^{-1}: the first k_c columns of Z stay, R_c
// is kept on the host, and U_c c = Z_c (R_c^{-1} c).  Columns k_c .. kr-1
// (kr = max k_c) are zero.  Returns kr.
static int build_recycle(Gmres32Work& G, const HostArnoldi& ha, int nrhs, int64_t ldv, int64_t ldz, cudaStream_t s) {
  const int64_t ldn = G.ldn;
  int kr = 0;
  for (int c = 0; c < nrhs; ++c) kr = std::max(kr, ha.jc[c]);
  if (kr <= 0) return 0;
  using cd = std::complex<double>;
  const size_t qsz = size_t(kr + 1) * kr, rsz = size_t(kr) * kr;
  std::vector<cd> Q(qsz);
  // per rhs: Q (column-major, leading dimension kr + 1) to the device, R kept on the host
  std::vector<float> q32(size_t(nrhs) * qsz * 2, 0.f);
  G.rec_R.assign(size_t(nrhs), std::vector<cd>());
  G.rec_kc.assign(size_t(nrhs), 0);
  for (int c = 0; c < nrhs; ++c) {
    const int kc = ha.jc[c];
    G.rec_kc[size_t(c)] = std::max(kc, 0);
    if (kc <= 0) continue;
    G.rec_R[size_t(c)].assign(rsz, cd(0));
    ha.qr(c, kc, Q.data(), G.rec_R[size_t(c)].data(), kr);
    float* qc = q32.data() + size_t(c) * qsz * 2;
    for (int p = 0; p < kc; ++p)
      for (int q = 0; q <= kc; ++q) {
        qc[2 * (size_t(p) * (kr + 1) + q)] = float(Q[size_t(p) * (kc + 1) + q].real());
        qc[2 * (size_t(p) * (kr + 1) + q) + 1] = float(Q[size_t(p) * (kc + 1) + q].imag());
      }
  }
  const size_t ncols = size_t(kr) * ldn * nrhs * 2;
  if (G.RC.n < ncols) G.RC.alloc(ncols);
  if (G.RQ.n < q32.size()) G.RQ.alloc(q32.size());
  MTF_CUDA(cudaMemcpyAsync(G.RQ.p, q32.data(), q32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  for (int c = 0; c < nrhs; ++c) {
    const int kc = ha.jc[c];
    float* Vc = G.V.p + 2 * size_t(c) * ldv;
    float* Zc = G.Z.p + 2 * size_t(c) * ldz;
    float* Cc = G.RC.p + 2 * size_t(c) * kr * ldn;
    const float* Qd = G.RQ.p + size_t(c) * qsz * 2;
    if (kc > 0) {
      // C = V Q over the first kc + 1 basis vectors
      const dim3 grid(unsigned((ldn + 127) / 128), unsigned((kc + 31) / 32));
      MTF_LAUNCH(KID_MISC, s, k_cgemm_nn<<<grid, 256, 0, s>>>(Vc, ldn, Qd, kr + 1, kc + 1, kc, ldn, Cc, ldn));
      MTF_CUDA(cudaMemcpyAsync(Vc, Cc, size_t(kc) * ldn * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (kc < kr) {
      MTF_CUDA(cudaMemsetAsync(Vc + 2 * size_t(kc) * ldn, 0, size_t(kr - kc) * ldn * 8, s));
      MTF_CUDA(cudaMemsetAsync(Zc + 2 * size_t(kc) * ldn, 0, size_t(kr - kc) * ldn * 8, s));
    }
  }
  MTF_CUDA(cudaStreamSynchronize(s));  // q32 is released on return
  return kr;
}

// the coefficients of the recycled columns (entries 0 .. kr-1 of each rhs's
// block of m + 1 complex values in yc) replaced by R_c^{-1} times them: back
// substitution with the kept upper-triangular factor
static void rec_coefficients(const Gmres32Work& G, std::vector<double>& yc, int nrhs, int m, int kr) {
  using cd = std::complex<double>;
  for (int c = 0; c < nrhs; ++c) {
    const int kc = G.rec_kc[size_t(c)];
    if (kc <= 0) continue;
    const std::vector<cd>& R = G.rec_R[size_t(c)];
    double* y = yc.data() + 2 * size_t(c) * (m + 1);
    for (int q = kc - 1; q >= 0; --q) {
      cd acc(y[2 * q], y[2 * q + 1]);
      for (int p = q + 1; p < kc; ++p) acc -= R[size_t(p) * kr + q] * cd(y[2 * p], y[2 * p + 1]);
      acc /= R[size_t(q) * kr + q];
      y[2 * q] = acc.real();
      y[2 * q + 1] = acc.imag();
    }
  }
}

mtf_status fgmres_cycle32(mtf_system sys, int nrhs, const double* r_dev, double* x_dev, double tol, int max_iter,
                          std::vector<int>& iters, bool& reached, cudaStream_t s, int cycle) {
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
    G.Z.alloc(size_t(m) * ldn * nrhs * 2);
    MTF_CUDA(cudaMemsetAsync(G.Z.p, 0, G.Z.n * sizeof(float), s));
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
    G.rec_k = 0;
  }
  if (cycle == 0) G.rec_k = 0;  // a new solve: nothing to recycle
  const int kr = G.rec_k;       // columns of the recycled space (0: none)
  G.rec_k = 0;                  // used by this cycle only
  const int ldh = m + 1;
  const int64_t ldv = int64_t(m + 1) * ldn, ldz = int64_t(m) * ldn;
  const size_t slot = slot_len(m - 1, nrhs);
  const dim3 ga{nb(ldn / 2, 32), unsigned(nrhs)};
  const dim3 gs{nb(ldn / 2, 256), unsigned(nrhs)};
  const size_t hsm = size_t(2 * m) * sizeof(float2);
  const size_t ysm = size_t(m + 1) * sizeof(double2);
  if (hsm > 40 * 1024 || ysm > 40 * 1024) {
    MTF_REQUIRE(ysm <= 200 * 1024 && hsm <= 200 * 1024, MTF_ERR_ARG,
                "restart length too large for the FP32 inner solver");
    MTF_CUDA(cudaFuncSetAttribute(k_axpy2_32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hsm) + 8192));
    MTF_CUDA(cudaFuncSetAttribute(k_xupdate32, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ysm)));
  }
  // x += sum_{i < jc[c]} Z_i y_i for coefficient vectors yc (m+1 complex per rhs)
  auto x_update = [&](const std::vector<double>& yc, const std::vector<int>& jcs) {
    int jm = 0;
    for (int c = 0; c < nrhs; ++c) jm = std::max(jm, jcs[size_t(c)]);
    if (jm <= 0) return;
    const size_t ny = yc.size();
    std::vector<double> ybuf(ny + size_t(nrhs));
    std::copy(yc.begin(), yc.end(), ybuf.begin());
    int* jp = reinterpret_cast<int*>(ybuf.data() + ny);
    for (int c = 0; c < nrhs; ++c) jp[c] = jcs[size_t(c)];
    if (G.y.n < ybuf.size()) G.y.alloc(ybuf.size());
    MTF_CUDA(cudaMemcpyAsync(G.y.p, ybuf.data(), ybuf.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    MTF_LAUNCH(KID_AXPY, s, k_xupdate32<<<ga, 256, size_t(jm) * sizeof(double2), s>>>(
        G.Z.p, G.y.p, reinterpret_cast<const int*>(G.y.p + ny), ldn, ldz, ldh, n, x_dev));
    MTF_CUDA(cudaStreamSynchronize(s));  // ybuf is released on return
  };

  HostArnoldi ha(m, nrhs);
  std::vector<int> active(nrhs);
  bool any = false;
  MTF_CUDA(cudaMemsetAsync(G.h.p, 0, size_t(nrhs) * sizeof(double), s));
  MTF_LAUNCH(KID_NORM, s, k_sqnorm64<<<dim3(nb(n, 256), unsigned(nrhs)), 256, 0, s>>>(r_dev, n, G.h.p));
  if (kr == 0) {
    // V_0 = r / ||r|| (sums of squares in slot 0)
    MTF_LAUNCH(KID_NORM, s, k_start32<<<dim3(nb(n, 256), unsigned(nrhs)), 256, 0, s>>>(r_dev, n, G.h.p, G.V.p, ldv));
    MTF_CUDA(cudaMemcpyAsync(G.h_host, G.h.p, size_t(nrhs) * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < nrhs; ++c) {
      const double rn = std::sqrt(G.h_host[c]);
      if (!std::isfinite(rn)) return MTF_ERR_NAN;
      ha.start(c, rn);
      active[c] = rn > 0;
      any = any || active[c];
    }
  } else {
    // Recycled start (GCRO): the residual is projected out of C = M U twice
    // (classical Gram-Schmidt), x += U (C^H r), and the new Krylov space
    // starts at column kr with the projected residual; the columns 0..kr-1
    // stay in the basis, so every later vector is also orthogonalised
    // against C.
    double* SS0 = G.h.p;                            // ||r||^2
    double* T1 = SS0 + nrhs;                        // C^H w, first pass
    double* S1 = T1 + 2 * size_t(kr) * nrhs;        // (unused second output of the dot kernel)
    double* T2 = S1 + 2 * size_t(kr) * nrhs;        // second pass
    double* SS1 = T2 + 2 * size_t(kr) * nrhs;       // ||w||^2 after pass 1 (unused), pass 2
    double* SS2 = SS1 + nrhs;
    double* NRM = SS2 + nrhs;
    const size_t used = size_t(NRM + 2 * nrhs - G.h.p);
    MTF_REQUIRE(used <= G.h.n, MTF_ERR_ARG, "recycled space larger than the Hessenberg scratch");
    MTF_CUDA(cudaMemsetAsync(T1, 0, (used - nrhs) * sizeof(double), s));
    MTF_LAUNCH(KID_NORM, s, k_start32<<<dim3(nb(n, 256), unsigned(nrhs)), 256, 0, s>>>(r_dev, n, SS0, G.w.p, ldn));
    launch_dots2_32(sys, G.V.p, G.w.p, ldn, ldv, kr, 0, T1, S1, nrhs, s);
    MTF_LAUNCH(KID_AXPY, s, k_proj32<<<ga, 256, 0, s>>>(G.V.p, T1, kr, nrhs, ldn, ldv, G.w.p, SS1));
    MTF_CUDA(cudaMemsetAsync(S1, 0, 2 * size_t(kr) * nrhs * sizeof(double), s));
    launch_dots2_32(sys, G.V.p, G.w.p, ldn, ldv, kr, 0, T2, S1, nrhs, s);
    MTF_LAUNCH(KID_AXPY, s, k_proj32<<<ga, 256, 0, s>>>(G.V.p, T2, kr, nrhs, ldn, ldv, G.w.p, SS2));
    MTF_LAUNCH(KID_NORM, s, k_scale32<<<gs, 256, 0, s>>>(G.w.p, ldn, SS2, NRM, G.V.p + 2 * size_t(kr) * ldn, ldv));
    MTF_CUDA(cudaMemcpyAsync(G.h_host, G.h.p, used * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    const double* hT1 = G.h_host + (T1 - G.h.p);
    const double* hT2 = G.h_host + (T2 - G.h.p);
    const double* hN = G.h_host + (NRM - G.h.p);
    std::vector<double> yc(size_t(m + 1) * nrhs * 2, 0.0);
    std::vector<int> jcs(nrhs, 0);
    for (int c = 0; c < nrhs; ++c) {
      const double rn = std::sqrt(G.h_host[c]);
      if (!std::isfinite(rn) || !std::isfinite(hN[2 * c])) return MTF_ERR_NAN;
      for (int i = 0; i < kr; ++i) {
        const size_t o = 2 * (size_t(i) * nrhs + c);
        yc[2 * (size_t(c) * (m + 1) + i)] = rn * (hT1[o] + hT2[o]);
        yc[2 * (size_t(c) * (m + 1) + i) + 1] = rn * (hT1[o + 1] + hT2[o + 1]);
      }
      jcs[c] = rn > 0 ? kr : 0;
      const double beta = rn * hN[2 * c];  // norm of the projected residual
      ha.start(c, beta, rn);
      active[c] = rn > 0 && beta > 0;
      any = any || active[c];
    }
    rec_coefficients(G, yc, nrhs, m, kr);
    x_update(yc, jcs);  // x += U (C^H r) = Z (R^{-1} C^H r)
  }
  reached = !any;
  if (!any) return MTF_OK;

  mtf_status status = MTF_OK;
  const int jend = std::min(m, kr + std::max(1, max_iter));
  // provisional (once-projected) column of every right-hand side, finished
  // when the next step's reduction arrives
  std::vector<std::vector<double>> rawcol(nrhs);
  std::vector<double> rawbeta(nrhs, 0.0);
  std::vector<double> hcol;
  // rows 0..kr-1 of the new columns (their components along C), per rhs
  std::vector<std::vector<double>> Bcol(nrhs);
  bool stop = false;
  auto finish_column = [&](int c, int jc, const double* sv, double alpha) -> double {
    // column jc with H[i, jc] += beta s_i (i <= jc) and H[jc+1, jc] = beta alpha
    hcol.assign(rawcol[c].begin(), rawcol[c].end());
    const double beta = rawbeta[c];
    if (sv)
      for (int i = 0; i <= jc; ++i) {
        hcol[2 * i] += beta * sv[2 * (size_t(i) * nrhs + c)];
        hcol[2 * i + 1] += beta * sv[2 * (size_t(i) * nrhs + c) + 1];
      }
    ++iters[c];
    if (kr > 0) Bcol[c].insert(Bcol[c].end(), hcol.begin(), hcol.begin() + 2 * size_t(kr));
    return ha.add_column(c, jc - kr, hcol.data() + 2 * size_t(kr), beta * alpha);
  };
  for (int j0 = kr; j0 < jend && !stop; j0 += kBatch) {
    const int nbat = std::min(kBatch, jend - j0);
    // the batch's Hessenberg slots are cleared once and copied back once
    MTF_CUDA(cudaMemsetAsync(G.h.p, 0, size_t(nbat) * slot * sizeof(double), s));
    for (int b = 0; b < nbat; ++b) {
      const int j = j0 + b;
      float* vj = G.V.p + 2 * size_t(j) * ldn;
      float* zj = G.Z.p + 2 * size_t(j) * ldn;
      if (pre) {
        launch_osrc_apply_f32(sys, vj, ldv, zj, ldz, nrhs, s);
        if (sys->learned_active) learned_apply_inplace(sys, vj, ldv, zj, ldz, nrhs, s);
      } else {
        MTF_CUDA(cudaMemcpy2DAsync(zj, size_t(ldz) * 8, vj, size_t(ldv) * 8, size_t(ldn) * 8, size_t(nrhs),
                                   cudaMemcpyDeviceToDevice, s));
      }
      launch_matvec_f32(sys, zj, ldz, G.w.p, ldn, nrhs, s);
      // delayed CGS2: one fused reduction, coefficients, one fused update
      double* T = G.h.p + size_t(b) * slot;
      double* S = T + 2 * size_t(j + 1) * nrhs;
      double* C = S + 2 * size_t(j + 1) * nrhs;
      double* NRM = C + 4 * size_t(nrhs);
      double* SS = NRM + 2 * size_t(nrhs);
      launch_dots2_32(sys, G.V.p, G.w.p, ldn, ldv, j + 1, j, T, S, nrhs, s);
      MTF_LAUNCH(KID_AXPY, s,
                 launch_pdl(k_axpy2_32, ga, dim3(256), size_t(2 * j) * sizeof(float2), s, G.V.p, T, S, C, j, kr,
                            nrhs, ldn, ldv, G.w.p, SS));
      MTF_LAUNCH(KID_NORM, s,
                 launch_pdl(k_scale32, gs, dim3(256), 0, s, G.w.p, ldn, SS, NRM, G.V.p + 2 * size_t(j + 1) * ldn,
                            ldv));
    }
    MTF_CUDA(cudaMemcpyAsync(G.h_host, G.h.p, (size_t(nbat - 1) * slot + slot_len(j0 + nbat - 1, nrhs)) * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < nbat && !stop; ++b) {
      const int j = j0 + b;
      const double* T = G.h_host + size_t(b) * slot;
      const double* S = T + 2 * size_t(j + 1) * nrhs;
      const double* C = S + 2 * size_t(j + 1) * nrhs;
      const double* NRM = C + 4 * size_t(nrhs);
      bool all_done = true;
      for (int c = 0; c < nrhs; ++c) {
        if (!active[c]) continue;
        if (j > kr) {
          const double alpha = C[2 * c];
          const double est = finish_column(c, j - 1, S, alpha);
          if (!std::isfinite(est)) status = MTF_ERR_NAN;
          if (est <= tol || rawbeta[c] * alpha == 0.0) active[c] = 0;
        }
        if (active[c]) {
          // provisional column j: t_0 .. t_{j-1}, h_j; subdiagonal ||w||
          rawcol[c].assign(2 * size_t(j + 1), 0.0);
          for (int i = 0; i < j; ++i) {
            rawcol[c][2 * i] = T[2 * (size_t(i) * nrhs + c)];
            rawcol[c][2 * i + 1] = T[2 * (size_t(i) * nrhs + c) + 1];
          }
          rawcol[c][2 * j] = C[2 * (nrhs + c)];
          rawcol[c][2 * j + 1] = C[2 * (nrhs + c) + 1];
          rawbeta[c] = NRM[2 * c];
        }
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
  if (!stop) {
    // cycle ended on its length: the last columns keep their once-projected values
    bool all_done = true;
    for (int c = 0; c < nrhs; ++c) {
      if (!active[c]) continue;
      const double est = finish_column(c, jend - 1, nullptr, 1.0);
      if (!std::isfinite(est)) status = MTF_ERR_NAN;
      if (est <= tol) active[c] = 0;
      all_done = all_done && !active[c];
    }
    if (all_done) reached = true;
    if (status != MTF_OK) {
      check_matvec_stream(sys, s);
      return status;
    }
  }
  check_matvec_stream(sys, s);
  // x += Z y, y = R^{-1} g per right-hand side (new columns); with a recycled
  // space also x -= U (B y), B the new columns' components along C
  std::vector<double> yhost(size_t(m + 1) * nrhs * 2);
  ha.solve(yhost);
  for (double v : yhost)
    if (!std::isfinite(v)) return MTF_ERR_NAN;
  std::vector<double> yc(size_t(m + 1) * nrhs * 2, 0.0);
  std::vector<int> jcs(nrhs, 0);
  for (int c = 0; c < nrhs; ++c) {
    const int jl = ha.jc[c];
    if (jl <= 0) continue;
    const double* yl = yhost.data() + 2 * size_t(c) * (m + 1);
    double* yo = yc.data() + 2 * size_t(c) * (m + 1);
    for (int q = 0; q < jl; ++q) {
      yo[2 * (kr + q)] = yl[2 * q];
      yo[2 * (kr + q) + 1] = yl[2 * q + 1];
    }
    for (int i = 0; i < kr; ++i) {
      double ur = 0, ui = 0;
      for (int q = 0; q < jl; ++q) {
        const double br = Bcol[c][2 * (size_t(q) * kr + i)], bi = Bcol[c][2 * (size_t(q) * kr + i) + 1];
        ur += br * yl[2 * q] - bi * yl[2 * q + 1];
        ui += br * yl[2 * q + 1] + bi * yl[2 * q];
      }
      yo[2 * i] = -ur;
      yo[2 * i + 1] = -ui;
    }
    jcs[c] = kr + jl;
  }
  if (kr > 0) rec_coefficients(G, yc, nrhs, m, kr);  // U (B y) = Z (R^{-1} B y)
  x_update(yc, jcs);
  // keep this cycle's space for the next cycle of the solve when there is
  // room for a useful number of new columns next to it
  if (cycle == 0 && kr == 0 && sys->opt.recycle) {
    int kmax = 0;
    for (int c = 0; c < nrhs; ++c) kmax = std::max(kmax, ha.jc[c]);
    if (kmax > 0 && kmax + 32 <= m) G.rec_k = build_recycle(G, ha, nrhs, ldv, ldz, s);
  }
  return status;
}

}  // namespace mtf
