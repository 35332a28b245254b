// Block flexible GMRES cycle of the mixed-precision inner solver: the nrhs
// right-hand sides of a solve share ONE Krylov space.  Block step j applies
// block-OSRC and the operator to the s = nrhs basis vectors together
// (Z_j = P V~_j, W = M Z_j), orthogonalises W against all earlier basis
// vectors by block classical Gram-Schmidt applied twice (BCGS2: the
// projections are skinny matrix products S = V^H X and X -= V S, on the
// tensor cores) and normalises it by a deflating Cholesky factorisation of
// its Gram matrix on the device.  The second Gram-Schmidt pass of a block is
// lagged by one step and shares the pass over the basis with the next
// block's first, so each step reads the basis twice (dots, update) instead
// of four times; the Hessenberg column block of step j is completed by step
// j + 1.  The block Hessenberg matrix is reduced by a progressive
// Householder QR on the host (block_krylov.h), which gives every right-hand
// side's residual estimate after each step; the update is x += Z Y with the
// least-squares coefficients Y.
//
// Why: at the same iteration count the block space is s times larger than
// each single-vector space, so a block step does the work of s single steps
// but the space grows toward every right-hand side at once.  For plane waves
// from many directions on the same scatterer the solve needs far fewer
// operator applies in total, and the Gram-Schmidt passes over the basis
// become products with s columns per basis read.
//
// Storage as in the single-vector cycle: complex FP32 vectors of padded
// length ldn (a multiple of 64, padding zero), vector-major; the Hessenberg
// coefficients are reduced in FP64 (FP64 atomics across CTAs).
#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "block_krylov.h"
#include "bulk.h"
#include "common.h"

namespace mtf {

struct TcArnoldi;
TcArnoldi* tca_create();
void tca_destroy(TcArnoldi* t);
void tca_set_dots_hi(TcArnoldi& t, bool on);
void tca_prepare(TcArnoldi& t, int s, int m, int64_t ldn, cudaStream_t st);
void tca_store(TcArnoldi& t, const float* Vn, int q0, cudaStream_t st);
void tca_project(TcArnoldi& t, int nq, float* W, int nc, double* H, int ldh, unsigned* err, cudaStream_t st);

struct BlockWork {
  int s = 0, m = 0;
  int64_t n = 0, ldn = 0;
  TcArnoldi* tca = nullptr;  // tensor-core projections (arnoldi_tc.cu), with mv_tensor
  DevBuf<float> V, Z, X, D;  // (m + 1) s, m s, 2 s ([V~_J | W]), s vectors
  DevBuf<double> S[2];       // projection coefficients of two steps: (m + 1) s x 2 s, complex
  DevBuf<double> Gs;         // Gpre (s) | G2 (2s x 2s) | G (s x s) | Hc ((m + 1) s x s) | Rn | R | Rv | Cc (two)
  DevBuf<double> C;          // s x s (complex, FP64) transform, or the coefficients Y (m s x s)
  DevBuf<int> kept;          // keptR (s) | keptV (s)
  double* h_host = nullptr;
  double* pin = nullptr;     // two pinned slots of a step's coefficients
  int* kept_host = nullptr;  // two pinned slots of kept flags and the error word
  cudaEvent_t ev[2] = {nullptr, nullptr};
  BlockLSQ lsq;
  ~BlockWork() {
    if (h_host) cudaFreeHost(h_host);
    if (pin) cudaFreeHost(pin);
    if (kept_host) cudaFreeHost(kept_host);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    tca_destroy(tca);
  }
};

void destroy_block32(BlockWork* w) { delete w; }

static inline unsigned nbk(int64_t n, int t) { return unsigned((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// H[q, c] += sum_k conj(V_q[k]) W_c[k] for q < nq, c < nc (<= SC): V_q at
// V + 2 q ldv, W_c at W + 2 c ldw (complex units); H complex FP64 at
// H + 2 (q ldh + c).  CTA: 8 warps x VW basis vectors, one segment of
// seg_len entries of the padded length n_pad, in chunks of 128 entries whose
// W slice is staged in shared memory; a lane takes entries 2 lane, 2 lane + 1,
// 64 + 2 lane, 65 + 2 lane of a chunk.  Sums over the lanes by recursive
// halving, then one FP64 atomic per (q, c, re / im) and segment.
// ---------------------------------------------------------------------------
template <int SC, int VW>
__global__ void __launch_bounds__(256) k_bdots(const float* __restrict__ V, int nq, int64_t ldv,
                                               const float* __restrict__ W, int64_t ldw, int nc, int64_t seg_len,
                                               int64_t n_pad, double* __restrict__ H, int ldh) {
  __shared__ __align__(16) float2 ws[SC][128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q0 = (int(blockIdx.y) * 8 + warp) * VW;
  const int64_t kb = int64_t(blockIdx.x) * seg_len;
  const int64_t ke = min(n_pad, kb + seg_len);
  constexpr int NV = VW * SC * 2;
  float acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0.f;
  for (int64_t k0 = kb; k0 < ke; k0 += 128) {
    __syncthreads();
    for (int t = threadIdx.x; t < SC * 64; t += 256) {
      const int c = t >> 6, e = t & 63;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < nc && k0 + 2 * e < ke) v = *reinterpret_cast<const float4*>(W + 2 * (int64_t(c) * ldw + k0 + 2 * e));
      *reinterpret_cast<float4*>(&ws[c][2 * e]) = v;
    }
    __syncthreads();
    float4 a0[VW], a1[VW];
    const bool second = k0 + 64 + 2 * lane < ke;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      a0[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      a1[v] = a0[v];
      if (q0 + v < nq) {
        const float* vb = V + 2 * (int64_t(q0 + v) * ldv + k0);
        if (k0 + 2 * lane < ke) a0[v] = *reinterpret_cast<const float4*>(vb + 4 * lane);
        if (second) a1[v] = *reinterpret_cast<const float4*>(vb + 128 + 4 * lane);
      }
    }
#pragma unroll
    for (int c = 0; c < SC; ++c) {
      const float4 w0 = *reinterpret_cast<const float4*>(&ws[c][2 * lane]);
      const float4 w1 = *reinterpret_cast<const float4*>(&ws[c][64 + 2 * lane]);
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        const float4 x = a0[v], y = a1[v];
        float re = acc[(v * SC + c) * 2], im = acc[(v * SC + c) * 2 + 1];
        re = fmaf(x.x, w0.x, re); re = fmaf(x.y, w0.y, re); re = fmaf(x.z, w0.z, re); re = fmaf(x.w, w0.w, re);
        re = fmaf(y.x, w1.x, re); re = fmaf(y.y, w1.y, re); re = fmaf(y.z, w1.z, re); re = fmaf(y.w, w1.w, re);
        im = fmaf(x.x, w0.y, im); im = fmaf(-x.y, w0.x, im); im = fmaf(x.z, w0.w, im); im = fmaf(-x.w, w0.z, im);
        im = fmaf(y.x, w1.y, im); im = fmaf(-y.y, w1.x, im); im = fmaf(y.z, w1.w, im); im = fmaf(-y.w, w1.z, im);
        acc[(v * SC + c) * 2] = re;
        acc[(v * SC + c) * 2 + 1] = im;
      }
    }
  }
  // lane sums: groups of 32 values, or one group of NV < 32 values
  if constexpr (NV >= 32) {
#pragma unroll
    for (int g = 0; g < NV / 32; ++g) {
      WarpTransposeSum<32>::run(acc + 32 * g, lane, 16);
      const int idx = 32 * g + lane;
      const int v = idx / (2 * SC), c = (idx >> 1) % SC;
      if (q0 + v < nq && c < nc) atomicAdd(H + 2 * (int64_t(q0 + v) * ldh + c) + (idx & 1), double(acc[32 * g]));
    }
  } else {
    WarpTransposeSum<NV>::run(acc, lane, 16);
    constexpr int SH = NV == 16 ? 1 : NV == 8 ? 2 : NV == 4 ? 3 : 4;
    if ((lane & ((1 << SH) - 1)) == 0) {
      const int idx = lane >> SH;
      const int v = idx / (2 * SC), c = (idx >> 1) % SC;
      if (q0 + v < nq && c < nc) atomicAdd(H + 2 * (int64_t(q0 + v) * ldh + c) + (idx & 1), double(acc[0]));
    }
  }
}

// ---------------------------------------------------------------------------
// W_c[k] -= sum_{q < nq} V_q[k] H[q, c] for c < nc (<= SC), H complex FP64 at
// H + 2 (q ldh + c), used in FP32.  CTA = 64 entries (a float4, two complex
// entries, per lane) x 8 warps over the basis vectors (q = warp mod 8); H is
// staged by chunks of 128 vectors, the 8 warps' partial sums are added in
// shared memory.
// ---------------------------------------------------------------------------
template <int SC>
__global__ void __launch_bounds__(256) k_bupdate(const float* __restrict__ V, int nq, int64_t ldv,
                                                 const double* __restrict__ H, int ldh, float* __restrict__ W,
                                                 int64_t ldw, int nc, int64_t n_pad) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  constexpr int QC = 128;
  __shared__ __align__(16) float2 hs[QC][SC];
  extern __shared__ __align__(16) float4 red[];  // [8][SC][32] float4 (two complex)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = int64_t(blockIdx.x) * 64 + 2 * lane;  // first of the lane's two entries
  const bool live = k < n_pad;
  float4 acc[SC];
#pragma unroll
  for (int c = 0; c < SC; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int qc = 0; qc < nq; qc += QC) {
    const int qn = min(QC, nq - qc);
    __syncthreads();
    for (int t = threadIdx.x; t < qn * SC; t += 256) {
      const int q = t / SC, c = t % SC;
      float2 h = make_float2(0.f, 0.f);
      if (c < nc) {
        const double* hp = H + 2 * (int64_t(qc + q) * ldh + c);
        h = make_float2(float(hp[0]), float(hp[1]));
      }
      hs[q][c] = h;
    }
    __syncthreads();
    if (live) {
      const float* vb = V + 2 * k;
#pragma unroll 4
      for (int q = warp; q < qn; q += 8) {
        const float4 a = *reinterpret_cast<const float4*>(vb + 2 * int64_t(qc + q) * ldv);
#pragma unroll
        for (int c = 0; c < SC; ++c) {
          const float2 h = hs[q][c];
          acc[c].x = fmaf(a.x, h.x, fmaf(-a.y, h.y, acc[c].x));
          acc[c].y = fmaf(a.x, h.y, fmaf(a.y, h.x, acc[c].y));
          acc[c].z = fmaf(a.z, h.x, fmaf(-a.w, h.y, acc[c].z));
          acc[c].w = fmaf(a.z, h.y, fmaf(a.w, h.x, acc[c].w));
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < SC; ++c) red[(warp * SC + c) * 32 + lane] = acc[c];
  __syncthreads();
  // warp w finishes columns c = w, w + 8, ...
  for (int c = warp; c < nc; c += 8) {
    float4 t = red[c * 32 + lane];
#pragma unroll
    for (int g = 1; g < 8; ++g) {
      const float4 p = red[(g * SC + c) * 32 + lane];
      t.x += p.x;
      t.y += p.y;
      t.z += p.z;
      t.w += p.w;
    }
    if (live) {
      float4* wp = reinterpret_cast<float4*>(W + 2 * (int64_t(c) * ldw + k));
      float4 o = *wp;
      o.x -= t.x;
      o.y -= t.y;
      o.z -= t.z;
      o.w -= t.w;
      *wp = o;
    }
  }
}

// out_q[k] = sum_{c < s} in_c[k] T[c, q] for q < s (T complex FP64, column-
// major s x s, used in FP32); thread per entry of the padded length
template <int SC>
__global__ void __launch_bounds__(256) k_bxform(const float* __restrict__ in, int64_t ldi, const double* __restrict__ T,
                                                int s, float* __restrict__ out, int64_t ldo, int64_t n_pad) {
  __shared__ float2 ts[SC][SC];
  for (int t = threadIdx.x; t < SC * SC; t += blockDim.x) {
    const int c = t / SC, q = t % SC;
    ts[c][q] = (c < s && q < s) ? make_float2(float(T[2 * (int64_t(q) * s + c)]), float(T[2 * (int64_t(q) * s + c) + 1]))
                                : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  float2 x[SC];
#pragma unroll
  for (int c = 0; c < SC; ++c) x[c] = c < s ? reinterpret_cast<const float2*>(in + 2 * int64_t(c) * ldi)[k] : make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < SC; ++q) {
    if (q >= s) break;
    float2 o = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < SC; ++c) {
      const float2 t = ts[c][q];
      o.x = fmaf(x[c].x, t.x, fmaf(-x[c].y, t.y, o.x));
      o.y = fmaf(x[c].x, t.y, fmaf(x[c].y, t.x, o.y));
    }
    reinterpret_cast<float2*>(out + 2 * int64_t(q) * ldo)[k] = o;
  }
}

// FP64 columns (stride n) -> FP32 columns (stride ldo, padded length, zero pad)
__global__ void k_blk_to32(const double* __restrict__ r, int64_t n, float* __restrict__ out, int64_t ldo) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= ldo) return;
  float2 v = make_float2(0.f, 0.f);
  if (k < n) {
    const double2 a = reinterpret_cast<const double2*>(r)[int64_t(c) * n + k];
    v = make_float2(float(a.x), float(a.y));
  }
  reinterpret_cast<float2*>(out + 2 * int64_t(c) * ldo)[k] = v;
}

// x_c (FP64, stride n) += d_c (FP32, stride ldd)
__global__ void k_blk_addx(double* __restrict__ x, int64_t n, const float* __restrict__ d, int64_t ldd) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 a = reinterpret_cast<const float2*>(d + 2 * int64_t(c) * ldd)[k];
  double2* xp = reinterpret_cast<double2*>(x) + int64_t(c) * n + k;
  double2 o = *xp;
  o.x += double(a.x);
  o.y += double(a.y);
  *xp = o;
}

// out[c] += ||W_c||^2 for the s columns of W (FP32 sums per thread and
// warp, one FP64 atomic per warp and column): the reference norms of the
// deflation test, read once from the block the operator just produced
__global__ void __launch_bounds__(256) k_bnorm2(const float* __restrict__ W, int64_t ldw, int64_t n,
                                                double* __restrict__ out) {
  const int c = blockIdx.y;
  const float4* w = reinterpret_cast<const float4*>(W + 2 * int64_t(c) * ldw);
  float a = 0.f;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n / 2; k += int64_t(gridDim.x) * blockDim.x) {
    const float4 v = w[k];  // two complex entries
    a = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, a))));
  }
  for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out + c, double(a));
}

// 1 / sqrt(d) for d > 0 in FP64: an FP32 seed refined by two Newton steps
// y <- y (3 - d y^2) / 2 (quadratic convergence: 2^-22 -> 2^-43 -> rounding);
// the narrow FP64 pipe makes this several times faster than sqrt and a
// division.  Outside the FP32 range the FP64 library functions are used.
__device__ __forceinline__ double rsqrt_newton(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = double(rsqrtf(float(d)));
  y = y * fma(-0.5 * d, y * y, 1.5);
  y = y * fma(-0.5 * d, y * y, 1.5);
  return y;
}

// Deflating Cholesky factor of a block's Gram matrix on the device (the
// rule of deflating_cholesky in block_krylov.h): G (complex FP64, entry
// [q ldg + c] = <W_q, W_c>) = R^H R with R upper triangular; direction k is
// dropped (row k of R zero, kept[k] = 0) when its Schur pivot is not above
// tau^2 ref_k, ref_k = ref[k] (squared norms before the
// Gram-Schmidt projections) or, with mask, 1 for mask[k] != 0 and 0
// otherwise.  R complex FP64, column-major (entry (i, c) at [c s + i]).
// One CTA of 256 threads, s <= 64: per pivot the row of R is formed in
// parallel and the trailing upper triangle is updated by all threads (the
// Schur complement and R in shared memory, s * s complex each).
//
// With C non-null (the second CholQR pass of V~_J), the same CTA then forms
// C = R^-H G_vw, the coordinates of W' along V_J = V~' R^-1, rows of dropped
// directions zero, from Gwv (Gwv[2 (c s + i)] = <W'_c, V~'_i>, so G_vw(i, c)
// = conj of it); C complex FP64 at C + 2 (i s + c), thread c solving
// column c from shared memory.
//
// T: the arithmetic.  FP64 for the first pass, whose pivots decide the
// deflation down to tau^2 = 1e-10 of a column's norm; FP32 for the second
// pass, whose Gram matrix is the identity to the FP32 rounding of the
// once-normalised block (its factor is I + O(2^-24) and FP32 keeps that),
// on the FP32 pipes instead of the narrow FP64 one.
template <class T>
struct CxOf;
template <>
struct CxOf<double> {
  using type = double2;
};
template <>
struct CxOf<float> {
  using type = float2;
};

__device__ __forceinline__ double rsqrt_of(double d) { return rsqrt_newton(d); }
__device__ __forceinline__ float rsqrt_of(float d) {
  const float y = rsqrtf(d);
  return y * fmaf(-0.5f * d, y * y, 1.5f);  // one Newton step on the approximate reciprocal square root
}

template <class T>
__global__ void __launch_bounds__(256) k_bchol(const double* __restrict__ G, int ldg, const double* __restrict__ ref,
                                               const int* __restrict__ mask, double tau, int s, double* __restrict__ R,
                                               int* __restrict__ kept, const double* __restrict__ Gwv,
                                               double* __restrict__ C) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  using T2 = typename CxOf<T>::type;
  extern __shared__ __align__(16) unsigned char shb[];
  T2* A = reinterpret_cast<T2*>(shb);  // A[c * s + i] = Schur complement entry (i, c), i <= c; then C
  T2* Rs = A + s * s;                  // Rs[c * s + i] = R(i, c)
  __shared__ T piv, ipiv, rinv[64];
  __shared__ double refs[64];
  __shared__ int keep, keeps[64];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < s * s; t += nt) {
    const int c = t / s, i = t % s;
    A[t] = T2{T(G[2 * (i * ldg + c)]), T(G[2 * (i * ldg + c) + 1])};
    Rs[t] = T2{T(0), T(0)};
  }
  for (int k = tid; k < s; k += nt) {
    refs[k] = mask ? (mask[k] ? 1.0 : 0.0) : ref[k];
    rinv[k] = T(0);
  }
  for (int k = 0; k < s; ++k) {
    __syncthreads();
    if (tid == 0) {
      const T d = A[k * s + k].x;
      keep = (double(d) > tau * tau * fmax(refs[k], 0.0) && d > T(0)) ? 1 : 0;
      if (keep) {
        const T y = rsqrt_of(d);
        piv = d * y;
        ipiv = y;
        rinv[k] = y;
      }
      keeps[k] = keep;
    }
    __syncthreads();
    if (!keep) continue;
    const T ip = ipiv;
    for (int c = k + tid; c < s; c += nt) {
      const T2 a = A[c * s + k];
      Rs[c * s + k] = c == k ? T2{piv, T(0)} : T2{a.x * ip, a.y * ip};
    }
    __syncthreads();
    const int w = s - k - 1;
    for (int t = tid; t < w * w; t += nt) {
      const int i = k + 1 + t % w, c = k + 1 + t / w;
      if (i > c) continue;
      const T2 ri = Rs[i * s + k], rc = Rs[c * s + k];  // R(k, i), R(k, c)
      A[c * s + i].x -= ri.x * rc.x + ri.y * rc.y;      // conj(R(k, i)) R(k, c)
      A[c * s + i].y -= ri.x * rc.y - ri.y * rc.x;
    }
  }
  __syncthreads();
  for (int t = tid; t < s * s; t += nt) {
    R[2 * t] = double(Rs[t].x);
    R[2 * t + 1] = double(Rs[t].y);
  }
  for (int k = tid; k < s; k += nt) kept[k] = keeps[k];
  if (C != nullptr && tid < s) {
    const int c = tid;
    T2* Cs = A;  // the Schur complement is no longer needed
    for (int i = 0; i < s; ++i) {
      T re = T(0), im = T(0);
      if (keeps[i]) {
        re = T(Gwv[2 * (c * s + i)]);    // G_vw(i, c) = conj(<W'_c, V~'_i>)
        im = -T(Gwv[2 * (c * s + i) + 1]);
        for (int p = 0; p < i; ++p) {  // - conj(R(p, i)) C[p, c]
          const T2 r = Rs[i * s + p], x = Cs[p * s + c];
          re -= r.x * x.x + r.y * x.y;
          im -= r.x * x.y - r.y * x.x;
        }
        re *= rinv[i];  // R(i, i) is real
        im *= rinv[i];
      }
      Cs[i * s + c] = T2{re, im};
      C[2 * (i * s + c)] = double(re);
      C[2 * (i * s + c) + 1] = double(im);
    }
  }
}

// out_q[k] = (in_q[k] - sum_{p < q} out_p[k] R(p, q)) / R(q, q) for kept q,
// 0 otherwise: V = W R^-1 on the kept set by forward substitution, entry by
// entry (R complex FP64, column-major, used in FP32)
template <int SC>
__global__ void __launch_bounds__(128) k_btrsm(const float* __restrict__ in, int64_t ldi, const double* __restrict__ R,
                                               const int* __restrict__ kept, int s, float* __restrict__ out, int64_t ldo,
                                               int64_t n_pad) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  __shared__ float2 rs[SC][SC];  // rs[p][q] = R(p, q)
  __shared__ float2 inv[SC];     // 1 / R(q, q), 0 for dropped q
  for (int t = threadIdx.x; t < SC * SC; t += blockDim.x) {
    const int p = t / SC, q = t % SC;
    rs[p][q] = (p < s && q < s) ? make_float2(float(R[2 * (q * s + p)]), float(R[2 * (q * s + p) + 1]))
                                : make_float2(0.f, 0.f);
  }
  for (int q = threadIdx.x; q < SC; q += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (q < s && kept[q]) {
      const double a = R[2 * (q * s + q)], b = R[2 * (q * s + q) + 1], d = a * a + b * b;
      v = make_float2(float(a / d), float(-b / d));
    }
    inv[q] = v;
  }
  __syncthreads();
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  float2 v[SC];
#pragma unroll
  for (int q = 0; q < SC; ++q) {
    if (q >= s) break;
    float2 a = reinterpret_cast<const float2*>(in + 2 * int64_t(q) * ldi)[k];
#pragma unroll
    for (int p = 0; p < q; ++p) {
      const float2 r = rs[p][q];
      a.x -= v[p].x * r.x - v[p].y * r.y;
      a.y -= v[p].x * r.y + v[p].y * r.x;
    }
    const float2 iv = inv[q];
    v[q] = make_float2(a.x * iv.x - a.y * iv.y, a.x * iv.y + a.y * iv.x);
    reinterpret_cast<float2*>(out + 2 * int64_t(q) * ldo)[k] = v[q];
  }
}

// k_btrsm for wide blocks (s > 16): the same forward substitution with the
// solved entries of each thread kept in shared memory instead of registers
// (SC complex values per thread would spill), R and the reciprocals staged
// as in k_btrsm.  Dynamic shared memory: SC^2 + SC x 128 complex FP32.
template <int SC>
__global__ void __launch_bounds__(128) k_btrsm_wide(const float* __restrict__ in, int64_t ldi,
                                                    const double* __restrict__ R, const int* __restrict__ kept, int s,
                                                    float* __restrict__ out, int64_t ldo, int64_t n_pad) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  extern __shared__ float2 shw[];
  float2* rs = shw;             // rs[p * SC + q] = R(p, q)
  float2* vs = shw + SC * SC;   // vs[q * 128 + thread]
  __shared__ float2 inv[SC];
  for (int t = threadIdx.x; t < SC * SC; t += blockDim.x) {
    const int p = t / SC, q = t % SC;
    rs[t] = (p < s && q < s) ? make_float2(float(R[2 * (q * s + p)]), float(R[2 * (q * s + p) + 1]))
                             : make_float2(0.f, 0.f);
  }
  for (int q = threadIdx.x; q < SC; q += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (q < s && kept[q]) {
      const double a = R[2 * (q * s + q)], b = R[2 * (q * s + q) + 1], d = a * a + b * b;
      v = make_float2(float(a / d), float(-b / d));
    }
    inv[q] = v;
  }
  __syncthreads();
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_pad) return;
  for (int q = 0; q < s; ++q) {
    float2 a = reinterpret_cast<const float2*>(in + 2 * int64_t(q) * ldi)[k];
    for (int p = 0; p < q; ++p) {
      const float2 r = rs[p * SC + q], v = vs[p * 128 + threadIdx.x];
      a.x -= v.x * r.x - v.y * r.y;
      a.y -= v.x * r.y + v.y * r.x;
    }
    const float2 iv = inv[q];
    const float2 o = make_float2(a.x * iv.x - a.y * iv.y, a.x * iv.y + a.y * iv.x);
    vs[q * 128 + threadIdx.x] = o;
    reinterpret_cast<float2*>(out + 2 * int64_t(q) * ldo)[k] = o;
  }
}

// R = the identity on the kept set (zero rows elsewhere), kept_out = kept_in:
// the start block of a cycle is already orthonormal (no lagged second pass)
__global__ void k_beye(const int* __restrict__ kept_in, int s, double* __restrict__ R, int* __restrict__ kept_out) {
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int c = t / s, i = t % s;
    R[2 * t] = (c == i && kept_in[i]) ? 1.0 : 0.0;
    R[2 * t + 1] = 0.0;
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) kept_out[i] = kept_in[i];
}

// C = R^-H G_vw on the kept set (rows of dropped directions zero): the
// coordinates of W' along V_J = V~' R^-1, from Gwv[2 (c s + i)] =
// <W'_c, V~'_i> (G_vw(i, c) is its conjugate).  C complex FP64 at
// C + 2 (i s + c), the layout of the update's coefficients.  R, G_vw and C
// are staged in shared memory (3 s^2 complex), the reciprocals of the
// diagonal of R^H are formed first, in parallel; then thread c runs the
// forward substitution of column c (no reductions across threads: the
// narrow FP64 pipe makes warp-shuffle sums the slower form).
__global__ void __launch_bounds__(64) k_bcoef(const double* __restrict__ Gwv, const double* __restrict__ R,
                                              const int* __restrict__ kept, int s, double* __restrict__ C) {
  extern __shared__ double2 sh[];
  double2* Rs = sh;              // Rs[i * s + p] = R(p, i)
  double2* Cs = sh + s * s;      // Cs[i * s + c]; first G_vw(i, c)
  __shared__ double2 rinv[64];   // 1 / conj(R(i, i)), 0 for dropped i
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    const int i = t / s, c = t % s;
    Rs[t] = make_double2(R[2 * t], R[2 * t + 1]);
    Cs[t] = make_double2(Gwv[2 * (c * s + i)], -Gwv[2 * (c * s + i) + 1]);  // conj(<W'_c, V~'_i>)
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (kept[i]) {
      const double dr = R[2 * (i * s + i)], di = R[2 * (i * s + i) + 1];
      const double dn = dr * dr + di * di;  // 1 / (dr - i di) = (dr + i di) / |d|^2
      v = make_double2(dr / dn, di / dn);
    }
    rinv[i] = v;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < s) {
    for (int i = 0; i < s; ++i) {
      double re = Cs[i * s + c].x, im = Cs[i * s + c].y;
      for (int p = 0; p < i; ++p) {  // - conj(R(p, i)) C[p, c]
        const double2 r = Rs[i * s + p], x = Cs[p * s + c];
        re -= r.x * x.x + r.y * x.y;
        im -= r.x * x.y - r.y * x.x;
      }
      const double2 ri = rinv[i];
      Cs[i * s + c] = make_double2(re * ri.x - im * ri.y, re * ri.y + im * ri.x);
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    C[2 * t] = Cs[t].x;
    C[2 * t + 1] = Cs[t].y;
  }
}

// Column block J - 1 of the block Hessenberg matrix, completed by step J
// (the second Gram-Schmidt pass of block J - 1's successor is lagged one
// step): with Sw = columns s .. 2s-1 of step J-1's coefficients, Sv =
// columns 0 .. s-1 of step J's (leading dimension 2 s both), C and R of
// step J - 1 and Rv of step J,
//   h[q, c] = Sw[q, c] + (Sv R)[q, c]            for q < nq0 = (J - 1) s,
//   h[q, c] = C[q - nq0, c] + (Sv R)[q, c]       for nq0 <= q < nq0 + s,
//   Rn = Rv R                                     (the subdiagonal block).
// h complex FP64 at h + 2 (q s + c); R, Rv, Rn column-major.  Thread (q, c).
__global__ void k_bhcol(const double* __restrict__ Sprev, const double* __restrict__ Scur,
                        const double* __restrict__ Cp, const double* __restrict__ Rp, const double* __restrict__ Rv,
                        int nq0, int s, double* __restrict__ h, double* __restrict__ Rn) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nh = int64_t(nq0 + s) * s;
  const int ls = 2 * s;
  if (t < nh) {
    const int q = int(t / s), c = int(t % s);
    double re, im;
    if (q < nq0) {
      re = Sprev[2 * (int64_t(q) * ls + s + c)];
      im = Sprev[2 * (int64_t(q) * ls + s + c) + 1];
    } else {
      re = Cp[2 * ((q - nq0) * s + c)];
      im = Cp[2 * ((q - nq0) * s + c) + 1];
    }
    // Sv holds the components V~_J kept along the earlier blocks after one
    // projection (about the FP32 rounding times the block's condition), so
    // its product with R is formed in FP32 and added to the FP64 part
    float cr = 0.f, ci = 0.f;
    for (int p = 0; p <= c; ++p) {  // R upper triangular: R(p, c) at [c s + p]
      const float ar = float(Scur[2 * (int64_t(q) * ls + p)]), ai = float(Scur[2 * (int64_t(q) * ls + p) + 1]);
      const float br = float(Rp[2 * (c * s + p)]), bi = float(Rp[2 * (c * s + p) + 1]);
      cr = fmaf(ar, br, fmaf(-ai, bi, cr));
      ci = fmaf(ar, bi, fmaf(ai, br, ci));
    }
    h[2 * t] = re + double(cr);
    h[2 * t + 1] = im + double(ci);
  } else if (t < nh + int64_t(s) * s) {
    const int u = int(t - nh), c = u / s, i = u % s;
    double re = 0.0, im = 0.0;
    for (int p = i; p <= c; ++p) {  // Rv(i, p) R(p, c)
      const double ar = Rv[2 * (p * s + i)], ai = Rv[2 * (p * s + i) + 1];
      const double br = Rp[2 * (c * s + p)], bi = Rp[2 * (c * s + p) + 1];
      re += ar * br - ai * bi;
      im += ar * bi + ai * br;
    }
    Rn[2 * (c * s + i)] = re;
    Rn[2 * (c * s + i) + 1] = im;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int col_tier(int s) { return s <= 1 ? 1 : s <= 2 ? 2 : s <= 4 ? 4 : s <= 8 ? 8 : 16; }

// H[q, c0 + c] += V_q^H W_{c0 + c} over all column groups of 16
static void bdots(mtf_system sys, const float* V, int nq, int64_t ldv, const float* W, int64_t ldw, int s, int64_t n_pad,
                  double* H, int ldh, cudaStream_t st, int kid = KID_BGRAM) {
  (void)sys;
  if (nq <= 0) return;
  for (int c0 = 0; c0 < s; c0 += 16) {
    const int nc = std::min(16, s - c0);
    const int SC = col_tier(nc);
    const int VW = SC >= 16 ? 2 : 4;
    const int gy = (nq + 8 * VW - 1) / (8 * VW);
    // segments so that about 600 CTAs run (fewer, longer segments measured
    // slower: 29 against 18 us for a 16-column Gram matrix of 72,000 entries)
    const int64_t nseg0 = std::max<int64_t>(1, std::min<int64_t>((n_pad + 127) / 128, (600 + gy - 1) / gy));
    const int64_t seg = ((n_pad + nseg0 - 1) / nseg0 + 127) / 128 * 128;
    const dim3 grid(unsigned((n_pad + seg - 1) / seg), unsigned(gy));
    const float* Wc = W + 2 * int64_t(c0) * ldw;
    double* Hc = H + 2 * c0;
    // basis and block read once
    prof_bytes(kid, double(nq + nc) * double(n_pad) * 8.0);
#define MTF_BDOTS(SCV, VWV) \
  MTF_LAUNCH(kid, st, k_bdots<SCV, VWV><<<grid, 256, 0, st>>>(V, nq, ldv, Wc, ldw, nc, seg, n_pad, Hc, ldh))
    if (SC == 16) MTF_BDOTS(16, 2);
    else if (SC == 8) MTF_BDOTS(8, 4);
    else if (SC == 4) MTF_BDOTS(4, 4);
    else if (SC == 2) MTF_BDOTS(2, 4);
    else MTF_BDOTS(1, 4);
#undef MTF_BDOTS
  }
}

template <int SC>
static void bupdate_launch(const float* V, int nq, int64_t ldv, const double* H, int ldh, float* W, int64_t ldw, int nc,
                           int64_t n_pad, int kid, cudaStream_t st) {
  const size_t smem = size_t(8) * SC * 32 * sizeof(float4);
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (smem > 48 * 1024 && !(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_bupdate<SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    opted.fetch_or(bit);
  }
  // basis read once, block read and written once
  prof_bytes(kid, double(nq + 2 * nc) * double(n_pad) * 8.0);
  MTF_LAUNCH(kid, st, launch_pdl(k_bupdate<SC>, dim3(nbk(n_pad, 64)), dim3(256), smem, st,
      V, nq, ldv, H, ldh, W, ldw, nc, n_pad));
}

// W_{c0 + c} -= sum_q V_q H[q, c0 + c] over all column groups of 16
// W -= V H over nq basis columns (kid: the profile entry; the Gram-Schmidt
// update of the FMA path counts as such, the small per-step corrections and
// the solution update as block transforms)
static void bupdate(const float* V, int nq, int64_t ldv, const double* H, int ldh, float* W, int64_t ldw, int s,
                    int64_t n_pad, cudaStream_t st, int kid = KID_BXFORM) {
  if (nq <= 0) return;
  for (int c0 = 0; c0 < s; c0 += 16) {
    const int nc = std::min(16, s - c0);
    const int SC = col_tier(nc);
    float* Wc = W + 2 * int64_t(c0) * ldw;
    const double* Hc = H + 2 * c0;
    if (SC == 16) bupdate_launch<16>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, kid, st);
    else if (SC == 8) bupdate_launch<8>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, kid, st);
    else if (SC == 4) bupdate_launch<4>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, kid, st);
    else if (SC == 2) bupdate_launch<2>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, kid, st);
    else bupdate_launch<1>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, kid, st);
  }
}

static void bxform(const float* in, int64_t ldi, const double* T, int s, float* out, int64_t ldo, int64_t n_pad,
                   cudaStream_t st) {
  const unsigned g = nbk(n_pad, 128);
#define MTF_BX(SCV) MTF_LAUNCH(KID_BXFORM, st, k_bxform<SCV><<<g, 128, 0, st>>>(in, ldi, T, s, out, ldo, n_pad))
  if (s <= 1) MTF_BX(1);
  else if (s <= 2) MTF_BX(2);
  else if (s <= 4) MTF_BX(4);
  else if (s <= 8) MTF_BX(8);
  else if (s <= 16) MTF_BX(16);
  else if (s <= 32) MTF_BX(32);
  else MTF_BX(64);
#undef MTF_BX
}

static void btrsm(const float* in, int64_t ldi, const double* R, const int* kept, int s, float* out, int64_t ldo,
                  int64_t n_pad, cudaStream_t st) {
  const unsigned g = nbk(n_pad, 128);
#define MTF_BT(SCV) \
  MTF_LAUNCH(KID_BXFORM, st, launch_pdl(k_btrsm<SCV>, dim3(g), dim3(128), 0, st, in, ldi, R, kept, s, out, ldo, n_pad))
  if (s <= 1) MTF_BT(1);
  else if (s <= 2) MTF_BT(2);
  else if (s <= 4) MTF_BT(4);
  else if (s <= 8) MTF_BT(8);
  else if (s <= 16) MTF_BT(16);
  else {
    // wide blocks: solved entries in shared memory
    const int SC = s <= 32 ? 32 : 64;
    const size_t smem = size_t(SC) * SC * sizeof(float2) + size_t(SC) * 128 * sizeof(float2);
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(opted.load() & bit)) {
      MTF_CUDA(cudaFuncSetAttribute(k_btrsm_wide<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(32 * 32 * 8 + 32 * 128 * 8)));
      MTF_CUDA(cudaFuncSetAttribute(k_btrsm_wide<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(64 * 64 * 8 + 64 * 128 * 8)));
      opted.fetch_or(bit);
    }
    if (SC == 32)
      MTF_LAUNCH(KID_BXFORM, st, launch_pdl(k_btrsm_wide<32>, dim3(g), dim3(128), smem, st,
          in, ldi, R, kept, s, out, ldo, n_pad));
    else
      MTF_LAUNCH(KID_BXFORM, st, launch_pdl(k_btrsm_wide<64>, dim3(g), dim3(128), smem, st,
          in, ldi, R, kept, s, out, ldo, n_pad));
  }
#undef MTF_BT
}

// G (nc x nc, complex FP64, G[a ldg + c] = <X_a, X_c>) of nc columns of
// stride ldx over n_pad entries (bdots: FP32 products per segment, FP64
// atomics; a two-stage kernel with per-CTA partial matrices measured slower,
// its shared-memory loads per product outweighing the saved atomics)
static void bgram(mtf_system sys, const float* X, int64_t ldx, int nc, int64_t n_pad, double* G, int ldg,
                  cudaStream_t st) {
  MTF_CUDA(cudaMemsetAsync(G, 0, 2 * size_t(nc) * ldg * sizeof(double), st));
  bdots(sys, X, nc, ldx, X, ldx, nc, n_pad, G, ldg, st);
}

// relative size below which a new direction of a block is deflated (its norm
// after orthogonalisation against the basis over its norm before): about a
// hundred times the FP32 rounding of the basis, so that the directions kept
// stay orthogonal to the basis to about 1e-2 after normalisation
constexpr double kDeflateTau = 1e-5;

mtf_status fgmres_block32(mtf_system sys, int s, const double* r_dev, double* x_dev, double tol, int max_iter,
                          std::vector<int>& iters, bool& reached, cudaStream_t st) {
  MTF_REQUIRE(s >= 1 && s <= 64, MTF_ERR_ARG, "block FGMRES supports 1..64 right-hand sides");
  mtf_mesh msh = sys->mesh;
  const int64_t n = msh->n_total;
  const int64_t ldn = (n + 63) & ~int64_t(63);
  const int m = std::max(1, sys->opt.restart);
  const bool pre = sys->opt.precond == MTF_PRECOND_OSRC;
  if (!sys->bw) sys->bw = new BlockWork();
  BlockWork& B = *sys->bw;
  stream_prepare(sys, st);  // error word of the bounded waits
  const size_t nhc = size_t(m + 1) * s * s;  // complex entries of a Hessenberg column block
  const size_t gsz = size_t(2) * (size_t(s) * s + 4 * size_t(s) * s + size_t(s) * s + nhc + 5 * size_t(s) * s);
  // pinned slot of a step (doubles): column block (nhc complex) | Rn (s x s complex)
  const size_t slot_len = 2 * nhc + 2 * size_t(s) * s;
  if (B.s != s || B.m != m || B.n != n) {
    B.V.alloc(size_t(m + 1) * s * ldn * 2);
    B.Z.alloc(size_t(m) * s * ldn * 2);
    B.X.alloc(size_t(2) * s * ldn * 2);
    B.D.alloc(size_t(s) * ldn * 2);
    MTF_CUDA(cudaMemsetAsync(B.V.p, 0, B.V.n * sizeof(float), st));
    MTF_CUDA(cudaMemsetAsync(B.Z.p, 0, B.Z.n * sizeof(float), st));
    MTF_CUDA(cudaMemsetAsync(B.X.p, 0, B.X.n * sizeof(float), st));
    for (auto& b : B.S) b.alloc(size_t(2) * (m + 1) * s * 2 * s);
    B.Gs.alloc(gsz);
    B.C.alloc(size_t(2) * std::max<size_t>(size_t(s) * s, size_t(m) * s * s));
    B.kept.alloc(size_t(2) * s);
    if (B.h_host) cudaFreeHost(B.h_host);
    if (B.pin) cudaFreeHost(B.pin);
    if (B.kept_host) cudaFreeHost(B.kept_host);
    B.h_host = nullptr;
    B.pin = nullptr;
    B.kept_host = nullptr;
    MTF_CUDA(cudaMallocHost(&B.h_host, 2 * size_t(s) * s * sizeof(double)));
    MTF_CUDA(cudaMallocHost(&B.pin, 2 * slot_len * sizeof(double)));
    MTF_CUDA(cudaMallocHost(&B.kept_host, 2 * (2 * size_t(s) + 1) * sizeof(int)));
    for (auto& e : B.ev)
      if (!e) MTF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B.s = s;
    B.m = m;
    B.n = n;
    B.ldn = ldn;
  }
  double* Gpre = B.Gs.p;                       // s: squared column norms of W before the projections
  double* G2 = Gpre + 2 * size_t(s) * s;       // 2s x s: <X_q, V~'_c> for the columns q of [V~', W']
  double* G = G2 + 8 * size_t(s) * s;          // s x s: Gram of W''
  double* Hc = G + 2 * size_t(s) * s;          // completed column block ((m + 1) s x s)
  double* Rn = Hc + 2 * nhc;                   // its subdiagonal block
  double* R = Rn + 2 * size_t(s) * s;          // W'' = V~_{J+1} R
  double* Rv = R + 2 * size_t(s) * s;          // V~' = V_J Rv
  double* CcBuf[2] = {Rv + 2 * size_t(s) * s, Rv + 4 * size_t(s) * s};  // W' = V_J Cc + W'' (steps by parity)
  int* keptR = B.kept.p;
  int* keptV = keptR + s;
  const int64_t vstride = int64_t(s) * ldn;  // complex entries per block of s vectors
  float* X0 = B.X.p;                          // V~_J (then V~')
  float* X1 = B.X.p + 2 * vstride;            // W (then W', W'')
  std::vector<cdouble> Gh(size_t(s) * s), R0(size_t(s) * s), T(size_t(s) * s);
  std::vector<double> Tup(size_t(2) * s * s), est(s, 0.0);
  std::vector<int> kept;
  // the Gram-Schmidt projections run on the tensor cores with the matvec
  const bool tc = sys->opt.mv_tensor != 0;
  if (tc) {
    if (!B.tca) B.tca = tca_create();
    tca_prepare(*B.tca, s, m, ldn, st);
    tca_set_dots_hi(*B.tca, sys->opt.gs_dots_half != 0);
  }
  unsigned* err_word = sys->d_mv_ctl.p + 2;
  // X[:, 0 .. nc) -= V S and S = V^H X against the first nq basis vectors (S leading dimension 2 s)
  auto project = [&](int nq, int nc, double* S) {
    if (tc) {
      tca_project(*B.tca, nq, B.X.p, nc, S, 2 * s, err_word, st);
    } else {
      MTF_CUDA(cudaMemsetAsync(S, 0, 2 * size_t(nq) * 2 * s * sizeof(double), st));
      bdots(sys, B.V.p, nq, ldn, B.X.p, ldn, nc, ldn, S, 2 * s, st, KID_DOTS);
      bupdate(B.V.p, nq, ldn, S, 2 * s, B.X.p, ldn, nc, ldn, st, KID_AXPY);
    }
  };

  // the residual block: X1 = r (FP32), its Gram matrix (norms ||r_c||) and
  // the start block V_0 = r T by the host's deflating Cholesky factor
  MTF_LAUNCH(KID_NORM, st, k_blk_to32<<<dim3(nbk(ldn, 256), unsigned(s)), 256, 0, st>>>(r_dev, n, X1, ldn));
  MTF_CUDA(cudaMemsetAsync(G, 0, 2 * size_t(s) * s * sizeof(double), st));
  bdots(sys, X1, s, ldn, X1, ldn, s, ldn, G, s, st);
  MTF_CUDA(cudaMemcpyAsync(B.h_host, G, 2 * size_t(s) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
  MTF_CUDA(cudaStreamSynchronize(st));
  // device layout [q * s + c] = <W_q, W_c>; column-major G[c * s + q] equals it
  for (int q = 0; q < s; ++q)
    for (int c = 0; c < s; ++c)
      Gh[size_t(c) * s + q] = cdouble(B.h_host[2 * (size_t(q) * s + c)], B.h_host[2 * (size_t(q) * s + c) + 1]);
  std::vector<double> bnorm(s), ref0(s);
  for (int c = 0; c < s; ++c) {
    const double d = Gh[size_t(c) * s + c].real();
    if (!std::isfinite(d)) return MTF_ERR_NAN;
    bnorm[c] = std::sqrt(std::max(d, 0.0));
    ref0[c] = d;
  }
  BlockLSQ& lsq = B.lsq;
  {
    // dependent or zero residual columns are deflated from the start
    const int nk0 = deflating_cholesky(s, Gh.data(), ref0.data(), 1e-12, R0.data(), T.data(), kept);
    reached = nk0 == 0;
    if (reached) return MTF_OK;
    for (size_t t = 0; t < T.size(); ++t) {
      Tup[2 * t] = T[t].real();
      Tup[2 * t + 1] = T[t].imag();
    }
    MTF_CUDA(cudaMemcpyAsync(B.C.p, Tup.data(), Tup.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    bxform(X1, ldn, B.C.p, s, B.V.p, ldn, ldn, st);
    if (tc) tca_store(*B.tca, B.V.p, 0, st);
    MTF_CUDA(cudaMemcpyAsync(keptR, kept.data(), size_t(s) * sizeof(int), cudaMemcpyHostToDevice, st));
    MTF_CUDA(cudaStreamSynchronize(st));  // T and kept are host memory
    lsq.init(s, m, R0.data(), bnorm.data());
  }

  // Pipelined block steps with the second Gram-Schmidt pass lagged by one
  // step.  Step J applies block-OSRC and the operator to V~_J, the block
  // orthogonalised once against the basis and normalised (Z_J = P V~_J,
  // W = M Z_J), and then, in ONE pass over the basis blocks 0 .. J - 1,
  // projects both V~_J (its second pass) and W (its first):
  //   [V~', W'] = [V~_J, W] - V [Sv, Sw].
  // V~' = V_J Rv (Cholesky of its Gram, the second CholQR pass) gives the
  // final block V_J; W' = V_J Cc + W'' (Cc = Rv^-H V~'^H W') and
  // W'' = V~_{J+1} R (Cholesky) the next lagged block.  Since
  // V~_J = V Sv + V_J Rv, column block J - 1 of the Hessenberg matrix,
  // M Z_{J-1} = V [Sw; Cc] + V~_J R, is completed by step J (k_bhcol).
  // Every kernel of a step runs on the device; its column block and kept
  // flags go to a pinned slot, and the host queues step J + 1 before it
  // reads step J's slot, so the least-squares update overlaps the device.
  // The last step of a cycle only finishes V~ (no operator apply).  A step
  // computed past convergence is discarded.  The basis holds m + 1 blocks
  // and Z holds m.
  const int Jend = std::min(m, std::max(1, max_iter));  // column blocks of this cycle
  {
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(opted.load() & bit)) {
      MTF_CUDA(cudaFuncSetAttribute(k_bchol<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 16));
      MTF_CUDA(cudaFuncSetAttribute(k_bchol<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 8));
      MTF_CUDA(cudaFuncSetAttribute(k_bcoef, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 16));
      opted.fetch_or(bit);
    }
  }
  const size_t chol_smem = 2 * size_t(s) * s * sizeof(double2), chol_smem32 = 2 * size_t(s) * s * sizeof(float2);
  auto slot = [&](int J) { return B.pin + size_t(J & 1) * slot_len; };
  auto launch_step = [&](int J) {
    const bool finish = J == Jend;
    double* Scur = B.S[J & 1].p;
    double* Cc = CcBuf[J & 1];
    const double* Cprev = CcBuf[(J + 1) & 1];
    const double* Sprev = B.S[(J + 1) & 1].p;
    float* Vt = B.V.p + 2 * int64_t(J) * vstride;  // V~_J; V_J after the step
    const int nq = J * s;
    const int nc = finish ? s : 2 * s;
    if (!finish) {
      float* Zj = B.Z.p + 2 * int64_t(J) * vstride;
      if (pre) {
        launch_osrc_apply_f32(sys, Vt, ldn, Zj, ldn, s, st);
        if (sys->learned_active) learned_apply_inplace(sys, Vt, ldn, Zj, ldn, s, st);
      } else {
        MTF_CUDA(cudaMemcpyAsync(Zj, Vt, size_t(s) * ldn * 8, cudaMemcpyDeviceToDevice, st));
      }
      launch_matvec_f32(sys, Zj, ldn, X1, ldn, s, st);
      MTF_CUDA(cudaMemsetAsync(Gpre, 0, size_t(s) * sizeof(double), st));
      MTF_LAUNCH(KID_BGRAM, st, k_bnorm2<<<dim3(64, unsigned(s)), 256, 0, st>>>(X1, ldn, ldn, Gpre));
    }
    MTF_CUDA(cudaMemcpyAsync(X0, Vt, size_t(s) * ldn * 8, cudaMemcpyDeviceToDevice, st));
    if (nq > 0) project(nq, nc, Scur);
    // <X_q, V~'_c> for every column q of X = [V~', W'] (G_vv, then the
    // conjugate of G_vw): one pass with s right-hand columns
    MTF_CUDA(cudaMemsetAsync(G2, 0, 2 * size_t(nc) * s * sizeof(double), st));
    bdots(sys, B.X.p, nc, ldn, X0, ldn, s, ldn, G2, s, st);
    const double* Gwv = G2 + 2 * size_t(s) * s;
    if (J == 0) {
      MTF_LAUNCH(KID_BCHOL, st, k_beye<<<1, 256, 0, st>>>(keptR, s, Rv, keptV));
    } else {
      // second CholQR pass of V~_J: directions that the first kept
      // Rv and, for a step with an operator apply, Cc = Rv^-H G_vw
      MTF_LAUNCH(KID_BCHOL, st, launch_pdl(k_bchol<float>, dim3(1), dim3(256), chol_smem32, st,
          G2, s, nullptr, keptR, 1e-3, s, Rv, keptV,
                                                                          Gwv, finish ? nullptr : Cc));
      MTF_LAUNCH(KID_BXFORM, st, launch_pdl(k_bhcol, dim3(nbk(int64_t(nq + s) * s, 256)), dim3(256), 0, st,
          Sprev, Scur, Cprev, R, Rv, nq - s, s, Hc, Rn));
    }
    if (!finish) {
      if (J > 0) btrsm(X0, ldn, Rv, keptV, s, Vt, ldn, ldn, st);
      // (step 0: V_0 is final, Cc = G_vw on its kept set)
      if (J == 0)
        MTF_LAUNCH(KID_BXFORM, st, k_bcoef<<<1, 64, 2 * size_t(s) * s * sizeof(double2), st>>>(Gwv, Rv, keptV, s, Cc));
      bupdate(Vt, s, ldn, Cc, s, X1, ldn, s, ldn, st);
      bgram(sys, X1, ldn, s, ldn, G, s, st);
      MTF_LAUNCH(KID_BCHOL, st, launch_pdl(k_bchol<double>, dim3(1), dim3(256), chol_smem, st,
          G, s, Gpre, nullptr, kDeflateTau, s, R,
                                                                           keptR, nullptr, nullptr));
      btrsm(X1, ldn, R, keptR, s, Vt + 2 * vstride, ldn, ldn, st);
      if (tc && J > 0) tca_store(*B.tca, Vt, J * s, st);
    }
    double* sl = slot(J);
    if (J > 0) {
      MTF_CUDA(cudaMemcpyAsync(sl, Hc, 2 * size_t(nq) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
      MTF_CUDA(cudaMemcpyAsync(sl + 2 * nhc, Rn, 2 * size_t(s) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    int* kh = B.kept_host + size_t(J & 1) * (2 * s + 1);
    MTF_CUDA(cudaMemcpyAsync(kh, keptR, 2 * size_t(s) * sizeof(int), cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(kh + 2 * s, err_word, sizeof(int), cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaEventRecord(B.ev[J & 1], st));
  };

  std::vector<cdouble> h, Rnh(size_t(s) * s);
  int steps = 0;
  mtf_status status = MTF_OK;
  using clk = std::chrono::steady_clock;
  auto since = [](clk::time_point a) { return std::chrono::duration<double>(clk::now() - a).count(); };
  auto tq = clk::now();
  launch_step(0);
  sys->t_launch += since(tq);
  for (int J = 0; J <= Jend; ++J) {
    tq = clk::now();
    if (J + 1 <= Jend) launch_step(J + 1);
    sys->t_launch += since(tq);
    tq = clk::now();
    MTF_CUDA(cudaEventSynchronize(B.ev[J & 1]));
    sys->t_wait += since(tq);
    const auto tl = clk::now();
    struct LsqClock {  // adds the host time of this step's update on every exit
      double& acc;
      clk::time_point t;
      ~LsqClock() { acc += std::chrono::duration<double>(clk::now() - t).count(); }
    } lsq_clock{sys->t_lsq, tl};
    const int* kh = B.kept_host + size_t(J & 1) * (2 * s + 1);
    if (kh[2 * s] != 0) {
      status = MTF_ERR_TIMEOUT;
      break;
    }
    if (J == 0) continue;
    // column block J - 1: rows of blocks 0 .. J - 1 and the subdiagonal block
    const double* sl = slot(J);
    const int nq = J * s;
    h.assign(size_t(nq) * s, cdouble(0));
    bool finite = true;
    for (int q = 0; q < nq; ++q)
      for (int c = 0; c < s; ++c) {
        const size_t o = 2 * (size_t(q) * s + c);
        const cdouble v(sl[o], sl[o + 1]);
        finite = finite && std::isfinite(v.real()) && std::isfinite(v.imag());
        h[size_t(c) * nq + q] = v;
      }
    for (size_t t = 0; t < size_t(s) * s; ++t) {
      Rnh[t] = cdouble(sl[2 * nhc + 2 * t], sl[2 * nhc + 2 * t + 1]);
      finite = finite && std::isfinite(Rnh[t].real()) && std::isfinite(Rnh[t].imag());
    }
    if (!finite) {
      status = MTF_ERR_NAN;
      break;
    }
    if (!lsq.add_block(h.data(), J, Rnh.data(), est.data())) break;
    ++steps;
    bool all = true;
    for (int c = 0; c < s; ++c) {
      if (!std::isfinite(est[c])) status = MTF_ERR_NAN;
      all = all && est[c] <= tol;
    }
    if (status != MTF_OK) break;
    if (all) {
      reached = true;
      break;
    }
    int nk = 0;  // directions of V_J
    for (int c = 0; c < s; ++c) nk += kh[s + c];
    if (nk == 0) break;  // the space is exhausted: the next cycle starts from the new residual
  }
  MTF_CUDA(cudaStreamSynchronize(st));  // a step queued past the last one has finished
  if (status != MTF_OK) {
    MTF_CUDA(cudaMemsetAsync(sys->d_mv_ctl.p, 0, 4 * sizeof(unsigned), st));
    return status;
  }
  for (int c = 0; c < s; ++c) iters[c] += steps;
  // x += Z Y over every column block of the space: D = 0 - Z (-Y)
  std::vector<cdouble> Y;
  lsq.solve(Y);
  const int nqz = lsq.k * s;
  if (nqz > 0) {
    std::vector<double> Yup(size_t(2) * nqz * s);
    for (int q = 0; q < nqz; ++q)
      for (int c = 0; c < s; ++c) {
        const cdouble v = Y[size_t(c) * nqz + q];
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return MTF_ERR_NAN;
        Yup[2 * (size_t(q) * s + c)] = -v.real();
        Yup[2 * (size_t(q) * s + c) + 1] = -v.imag();
      }
    MTF_CUDA(cudaMemcpyAsync(B.C.p, Yup.data(), Yup.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    MTF_CUDA(cudaMemsetAsync(B.D.p, 0, B.D.n * sizeof(float), st));
    bupdate(B.Z.p, nqz, ldn, B.C.p, s, B.D.p, ldn, s, ldn, st);
    MTF_LAUNCH(KID_AXPY, st, k_blk_addx<<<dim3(nbk(n, 256), unsigned(s)), 256, 0, st>>>(x_dev, n, B.D.p, ldn));
  }
  MTF_CUDA(cudaStreamSynchronize(st));  // host buffers are released on return
  return MTF_OK;
}

}  // namespace mtf
