// Block flexible GMRES cycle of the mixed-precision inner solver: the nrhs
// right-hand sides of a solve share ONE Krylov space.  Block step j applies
// block-OSRC and the operator to the s = nrhs basis vectors V_j together
// (Z_j = P V_j, W = M Z_j), orthogonalises W against all earlier basis
// vectors by block classical Gram-Schmidt applied twice (BCGS2: the
// projections are skinny matrix products H = V^H W and W -= V H), and
// normalises it by a deflating Cholesky factorisation of its Gram matrix
// (host, block_krylov.h), W = V_{j+1} R_{j+1}.  The block Hessenberg matrix
// is reduced by a progressive Householder QR on the host, which gives every
// right-hand side's residual estimate after each step; the update is
// x += Z Y with the least-squares coefficients Y.
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
void tca_prepare(TcArnoldi& t, int s, int m, int64_t ldn, cudaStream_t st);
void tca_store(TcArnoldi& t, const float* Vn, int q0, cudaStream_t st);
void tca_project(TcArnoldi& t, int nq, float* W, double* H, unsigned* err, cudaStream_t st);

struct BlockWork {
  int s = 0, m = 0;
  int64_t n = 0, ldn = 0;
  TcArnoldi* tca = nullptr;  // tensor-core projections (arnoldi_tc.cu), with mv_tensor
  DevBuf<float> V, Z, W, D;  // (m + 1) s, m s, s, s vectors
  DevBuf<double> H;          // Gpre (s x s) | H1 ((m+1) s x s) | H2 | G (s x s), complex
  DevBuf<double> C;          // s x s (complex, FP64) transform, or the coefficients Y (m s x s)
  DevBuf<double> Cd;         // R1, T1, R2, T2 of a step's Cholesky factorisations (complex s x s each)
  DevBuf<int> kept;          // kept flags of the two factorisations
  double* h_host = nullptr;
  double* pin = nullptr;     // two pinned slots of a step's coefficients
  int* kept_host = nullptr;  // two pinned slots of kept flags and the error word
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // the space of the solve's previous cycle, kept for the next one
  BlockLSQ lsq;
  bool rec_ok = false;
  int vshift = 0;
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

// Deflating Cholesky factor of a block's Gram matrix on the device (the
// rule of deflating_cholesky in block_krylov.h): G (complex FP64, entry
// [q s + c] = <W_q, W_c>) = R^H R with R upper triangular; direction k is
// dropped (row k of R zero, kept[k] = 0) when its Schur pivot is not above
// tau^2 ref_k, ref_k = the diagonal of Gpre (squared norms before the
// Gram-Schmidt projections) or, with mask, 1 for mask[k] != 0 and 0
// otherwise.  R complex FP64, column-major (entry (i, c) at [c s + i]).
// One CTA of 256 threads, s <= 64: per pivot the row of R is formed in
// parallel and the trailing upper triangle is updated by all threads (the
// Schur complement and R in shared memory, s * s complex each).
__global__ void __launch_bounds__(256) k_bchol(const double* __restrict__ G, const double* __restrict__ Gpre,
                                               const int* __restrict__ mask, double tau, int s, double* __restrict__ R,
                                               int* __restrict__ kept) {
  extern __shared__ double2 sh[];
  double2* A = sh;           // A[c * s + i] = Schur complement entry (i, c), i <= c
  double2* Rs = sh + s * s;  // Rs[c * s + i] = R(i, c)
  __shared__ double piv;
  __shared__ int keep;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < s * s; t += nt) {
    const int c = t / s, i = t % s;
    A[t] = make_double2(G[2 * (i * s + c)], G[2 * (i * s + c) + 1]);
    Rs[t] = make_double2(0.0, 0.0);
  }
  for (int k = 0; k < s; ++k) {
    __syncthreads();
    if (tid == 0) {
      const double d = A[k * s + k].x;
      const double ref = mask ? (mask[k] ? 1.0 : 0.0) : Gpre[2 * (k * s + k)];
      keep = (d > tau * tau * fmax(ref, 0.0) && d > 0.0) ? 1 : 0;
      piv = keep ? sqrt(d) : 0.0;
      kept[k] = keep;
    }
    __syncthreads();
    if (!keep) continue;
    const double ip = 1.0 / piv;
    for (int c = k + tid; c < s; c += nt) {
      const double2 a = A[c * s + k];
      Rs[c * s + k] = c == k ? make_double2(piv, 0.0) : make_double2(a.x * ip, a.y * ip);
    }
    __syncthreads();
    const int w = s - k - 1;
    for (int t = tid; t < w * w; t += nt) {
      const int i = k + 1 + t % w, c = k + 1 + t / w;
      if (i > c) continue;
      const double2 ri = Rs[i * s + k], rc = Rs[c * s + k];  // R(k, i), R(k, c)
      A[c * s + i].x -= ri.x * rc.x + ri.y * rc.y;            // conj(R(k, i)) R(k, c)
      A[c * s + i].y -= ri.x * rc.y - ri.y * rc.x;
    }
  }
  __syncthreads();
  for (int t = tid; t < s * s; t += nt) {
    R[2 * t] = Rs[t].x;
    R[2 * t + 1] = Rs[t].y;
  }
}

// out_q[k] = (in_q[k] - sum_{p < q} out_p[k] R(p, q)) / R(q, q) for kept q,
// 0 otherwise: V = W R^-1 on the kept set by forward substitution, entry by
// entry (R complex FP64, column-major, used in FP32)
template <int SC>
__global__ void __launch_bounds__(128) k_btrsm(const float* __restrict__ in, int64_t ldi, const double* __restrict__ R,
                                               const int* __restrict__ kept, int s, float* __restrict__ out, int64_t ldo,
                                               int64_t n_pad) {
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int col_tier(int s) { return s <= 1 ? 1 : s <= 2 ? 2 : s <= 4 ? 4 : s <= 8 ? 8 : 16; }

// H[q, c0 + c] += V_q^H W_{c0 + c} over all column groups of 16
static void bdots(mtf_system sys, const float* V, int nq, int64_t ldv, const float* W, int64_t ldw, int s, int64_t n_pad,
                  double* H, int ldh, cudaStream_t st) {
  (void)sys;
  if (nq <= 0) return;
  for (int c0 = 0; c0 < s; c0 += 16) {
    const int nc = std::min(16, s - c0);
    const int SC = col_tier(nc);
    const int VW = SC >= 16 ? 2 : 4;
    const int gy = (nq + 8 * VW - 1) / (8 * VW);
    // segments so that about 600 CTAs run
    const int64_t nseg0 = std::max<int64_t>(1, std::min<int64_t>((n_pad + 127) / 128, (600 + gy - 1) / gy));
    const int64_t seg = ((n_pad + nseg0 - 1) / nseg0 + 127) / 128 * 128;
    const dim3 grid(unsigned((n_pad + seg - 1) / seg), unsigned(gy));
    const float* Wc = W + 2 * int64_t(c0) * ldw;
    double* Hc = H + 2 * c0;
    // basis and block read once
    prof_bytes(KID_DOTS, double(nq + nc) * double(n_pad) * 8.0);
#define MTF_BDOTS(SCV, VWV) \
  MTF_LAUNCH(KID_DOTS, st, k_bdots<SCV, VWV><<<grid, 256, 0, st>>>(V, nq, ldv, Wc, ldw, nc, seg, n_pad, Hc, ldh))
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
                           int64_t n_pad, cudaStream_t st) {
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
  prof_bytes(KID_AXPY, double(nq + 2 * nc) * double(n_pad) * 8.0);
  MTF_LAUNCH(KID_AXPY, st, k_bupdate<SC><<<nbk(n_pad, 64), 256, smem, st>>>(V, nq, ldv, H, ldh, W, ldw, nc, n_pad));
}

// W_{c0 + c} -= sum_q V_q H[q, c0 + c] over all column groups of 16
static void bupdate(const float* V, int nq, int64_t ldv, const double* H, int ldh, float* W, int64_t ldw, int s,
                    int64_t n_pad, cudaStream_t st) {
  if (nq <= 0) return;
  for (int c0 = 0; c0 < s; c0 += 16) {
    const int nc = std::min(16, s - c0);
    const int SC = col_tier(nc);
    float* Wc = W + 2 * int64_t(c0) * ldw;
    const double* Hc = H + 2 * c0;
    if (SC == 16) bupdate_launch<16>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, st);
    else if (SC == 8) bupdate_launch<8>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, st);
    else if (SC == 4) bupdate_launch<4>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, st);
    else if (SC == 2) bupdate_launch<2>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, st);
    else bupdate_launch<1>(V, nq, ldv, Hc, ldh, Wc, ldw, nc, n_pad, st);
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
  MTF_LAUNCH(KID_BXFORM, st, k_btrsm<SCV><<<g, 128, 0, st>>>(in, ldi, R, kept, s, out, ldo, n_pad))
  if (s <= 1) MTF_BT(1);
  else if (s <= 2) MTF_BT(2);
  else if (s <= 4) MTF_BT(4);
  else if (s <= 8) MTF_BT(8);
  else if (s <= 16) MTF_BT(16);
  else if (s <= 32) MTF_BT(32);
  else MTF_BT(64);
#undef MTF_BT
}

// relative size below which a new direction of a block is deflated (its norm
// after orthogonalisation against the basis over its norm before): about a
// hundred times the FP32 rounding of the basis, so that the directions kept
// stay orthogonal to the basis to about 1e-2 after normalisation
constexpr double kDeflateTau = 1e-5;

// kept restarts in a row (each widens the least-squares band by one block)
constexpr int kMaxKeep = 2;

mtf_status fgmres_block32(mtf_system sys, int s, const double* r_dev, double* x_dev, double tol, int max_iter,
                          std::vector<int>& iters, bool& reached, cudaStream_t st, int cycle) {
  MTF_REQUIRE(s >= 1 && s <= 64, MTF_ERR_ARG, "block FGMRES supports 1..64 right-hand sides");
  mtf_mesh msh = sys->mesh;
  const int64_t n = msh->n_total;
  const int64_t ldn = (n + 63) & ~int64_t(63);
  const int m = std::max(1, sys->opt.restart);
  const bool pre = sys->opt.precond == MTF_PRECOND_OSRC;
  if (!sys->bw) sys->bw = new BlockWork();
  BlockWork& B = *sys->bw;
  stream_prepare(sys, st);  // error word of the bounded waits
  const size_t hsz = size_t(2) * (s * s + 2 * size_t(m + 1) * s * s + s * s);
  if (B.s != s || B.m != m || B.n != n) {
    B.V.alloc(size_t(m + 1) * s * ldn * 2);
    B.Z.alloc(size_t(m) * s * ldn * 2);
    B.W.alloc(size_t(s) * ldn * 2);
    B.D.alloc(size_t(s) * ldn * 2);
    MTF_CUDA(cudaMemsetAsync(B.V.p, 0, B.V.n * sizeof(float), st));
    MTF_CUDA(cudaMemsetAsync(B.Z.p, 0, B.Z.n * sizeof(float), st));
    MTF_CUDA(cudaMemsetAsync(B.W.p, 0, B.W.n * sizeof(float), st));
    B.H.alloc(hsz);
    B.C.alloc(size_t(2) * std::max<size_t>(size_t(s) * s, size_t(m) * s * s));
    B.Cd.alloc(size_t(8) * s * s);
    B.kept.alloc(size_t(2) * s);
    if (B.h_host) cudaFreeHost(B.h_host);
    if (B.pin) cudaFreeHost(B.pin);
    if (B.kept_host) cudaFreeHost(B.kept_host);
    B.h_host = nullptr;
    B.pin = nullptr;
    B.kept_host = nullptr;
    MTF_CUDA(cudaMallocHost(&B.h_host, hsz * sizeof(double)));
    const size_t slot_len = 4 * size_t(m + 1) * s * s + 4 * size_t(s) * s + 2 * size_t(s) + 1;
    MTF_CUDA(cudaMallocHost(&B.pin, 2 * slot_len * sizeof(double)));
    MTF_CUDA(cudaMallocHost(&B.kept_host, 2 * (2 * size_t(s) + 1) * sizeof(int)));
    for (auto& e : B.ev)
      if (!e) MTF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B.s = s;
    B.m = m;
    B.n = n;
    B.ldn = ldn;
    B.rec_ok = false;
  }
  double* Gpre = B.H.p;
  double* H1 = Gpre + 2 * size_t(s) * s;
  double* H2 = H1 + 2 * size_t(m + 1) * s * s;
  double* G = H2 + 2 * size_t(m + 1) * s * s;
  const int64_t vstride = int64_t(s) * ldn;  // complex entries per block of s vectors
  std::vector<cdouble> Gh(size_t(s) * s), R(size_t(s) * s), T(size_t(s) * s);
  std::vector<double> ref(s), Tup(size_t(2) * s * s), est(s, 0.0);
  std::vector<int> kept;
  auto fetch_gram = [&](const double* dev, std::vector<cdouble>& out) {
    // device layout [q * s + c] = <W_q, W_c>; column-major G[c * s + q] equals it
    for (int q = 0; q < s; ++q)
      for (int c = 0; c < s; ++c) {
        const double* p = B.h_host + (dev - B.H.p) + 2 * (size_t(q) * s + c);
        out[size_t(c) * s + q] = cdouble(p[0], p[1]);
      }
  };
  auto upload_T = [&](const std::vector<cdouble>& Tm) {
    for (size_t t = 0; t < Tm.size(); ++t) {
      Tup[2 * t] = Tm[t].real();
      Tup[2 * t + 1] = Tm[t].imag();
    }
    MTF_CUDA(cudaMemcpyAsync(B.C.p, Tup.data(), Tup.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  };
  // the Gram-Schmidt projections run on the tensor cores with the matvec
  const bool tc = sys->opt.mv_tensor != 0;
  if (tc) {
    if (!B.tca) B.tca = tca_create();
    tca_prepare(*B.tca, s, m, ldn, st);
  }
  unsigned* err_word = sys->d_mv_ctl.p + 2;
  const double tau = kDeflateTau;
  auto project = [&](int nq) {  // W <- (I - V V^H)^2 W against the first nq basis vectors; H1, H2 the coefficients
    if (tc) {
      tca_project(*B.tca, nq, B.W.p, H1, err_word, st);
      tca_project(*B.tca, nq, B.W.p, H2, err_word, st);
    } else {
      MTF_CUDA(cudaMemsetAsync(H1, 0, 2 * size_t(nq) * s * sizeof(double), st));
      MTF_CUDA(cudaMemsetAsync(H2, 0, 2 * size_t(nq) * s * sizeof(double), st));
      bdots(sys, B.V.p, nq, ldn, B.W.p, ldn, s, ldn, H1, s, st);
      bupdate(B.V.p, nq, ldn, H1, s, B.W.p, ldn, s, ldn, st);
      bdots(sys, B.V.p, nq, ldn, B.W.p, ldn, s, ldn, H2, s, st);
      bupdate(B.V.p, nq, ldn, H2, s, B.W.p, ldn, s, ldn, st);
    }
  };

  // the residual block: W = r (FP32) and its Gram matrix (norms ||r_c||)
  MTF_LAUNCH(KID_NORM, st, k_blk_to32<<<dim3(nbk(ldn, 256), unsigned(s)), 256, 0, st>>>(r_dev, n, B.W.p, ldn));
  MTF_CUDA(cudaMemsetAsync(G, 0, 2 * size_t(s) * s * sizeof(double), st));
  bdots(sys, B.W.p, s, ldn, B.W.p, ldn, s, ldn, G, s, st);
  MTF_CUDA(cudaMemcpyAsync(B.h_host + (G - B.H.p), G, 2 * size_t(s) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
  MTF_CUDA(cudaStreamSynchronize(st));
  fetch_gram(G, Gh);
  std::vector<double> bnorm(s), ref0(s);
  for (int c = 0; c < s; ++c) {
    const double d = Gh[size_t(c) * s + c].real();
    if (!std::isfinite(d)) return MTF_ERR_NAN;
    bnorm[c] = std::sqrt(std::max(d, 0.0));
    ref0[c] = d;
  }
  // Restart that keeps the space (the next refinement cycle of one solve):
  // the new residual is projected on the basis built so far, its remainder
  // opens a new start block, and the new column blocks are orthogonalised
  // against the whole basis, so the cycle does not rebuild the slow start
  // of the previous one.  Column block J then multiplies basis block
  // J + vshift (vshift = kept restarts so far).
  BlockLSQ& lsq = B.lsq;
  const int nb_old = lsq.k + 1 + B.vshift;
  const bool keep = cycle > 0 && sys->opt.recycle >= 2 && B.rec_ok && lsq.s == s && B.vshift < kMaxKeep &&
                    nb_old + 16 <= m;
  B.rec_ok = false;
  bool grow = true;  // the start block has a kept direction
  if (!keep) {
    // dependent or zero residual columns are deflated from the start
    const int nk0 = deflating_cholesky(s, Gh.data(), ref0.data(), 1e-12, R.data(), T.data(), kept);
    reached = nk0 == 0;
    if (reached) return MTF_OK;
    upload_T(T);
    bxform(B.W.p, ldn, B.C.p, s, B.V.p, ldn, ldn, st);
    if (tc) tca_store(*B.tca, B.V.p, 0, st);
    lsq.init(s, m, R.data(), bnorm.data(), 1 + kMaxKeep);
    B.vshift = 0;
  } else {
    const int nq_old = nb_old * s;
    project(nq_old);
    MTF_CUDA(cudaMemsetAsync(G, 0, 2 * size_t(s) * s * sizeof(double), st));
    bdots(sys, B.W.p, s, ldn, B.W.p, ldn, s, ldn, G, s, st);
    MTF_CUDA(cudaMemcpyAsync(B.h_host + (H1 - B.H.p), H1, 2 * size_t(nq_old) * s * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(B.h_host + (H2 - B.H.p), H2, 2 * size_t(nq_old) * s * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(B.h_host + (G - B.H.p), G, 2 * size_t(s) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaStreamSynchronize(st));
    fetch_gram(G, Gh);
    const int nk0 = deflating_cholesky(s, Gh.data(), ref0.data(), tau, R.data(), T.data(), kept);
    const size_t nr = size_t(nq_old + s);
    std::vector<cdouble> G0(nr * s);
    const double* hp1 = B.h_host + (H1 - B.H.p);
    const double* hp2 = B.h_host + (H2 - B.H.p);
    for (int c = 0; c < s; ++c) {
      for (int q = 0; q < nq_old; ++q) {
        const size_t o = 2 * (size_t(q) * s + c);
        G0[size_t(c) * nr + q] = cdouble(hp1[o] + hp2[o], hp1[o + 1] + hp2[o + 1]);
      }
      for (int i = 0; i < s; ++i) G0[size_t(c) * nr + nq_old + i] = R[size_t(c) * s + i];
    }
    for (const cdouble& v : G0)
      if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return MTF_ERR_NAN;
    upload_T(T);
    float* V0 = B.V.p + 2 * int64_t(nb_old) * vstride;
    bxform(B.W.p, ldn, B.C.p, s, V0, ldn, ldn, st);
    if (tc) tca_store(*B.tca, V0, nq_old, st);
    lsq.restart(G0.data(), nb_old + 1, bnorm.data(), est.data());
    B.vshift += 1;
    bool all = true;
    for (int c = 0; c < s; ++c) all = all && est[c] <= tol;
    reached = all;
    grow = !all && nk0 > 0;
  }
  const int vshift = B.vshift;
  const int J0 = lsq.k;

  // Pipelined block steps.  Everything of step J runs on the device --
  // block-OSRC, the matvec, both Gram-Schmidt projections, the deflating
  // Cholesky factorisations (two: CholQR2) and the next basis block -- and
  // its coefficients (H1, H2, R1, R2, the kept flags and the error word) are
  // copied to a pinned slot; the host queues step J + 1 before it reads step
  // J's slot, so that the least-squares update of step J overlaps the device
  // work of step J + 1.  A step computed past convergence is discarded.
  // Column block J multiplies basis block J + vshift and produces block
  // J + vshift + 1; the basis holds m + 1 blocks and Z holds m.
  const int Jend = std::min(m - vshift, J0 + std::max(1, max_iter));
  double* R1 = B.Cd.p;
  double* R2 = R1 + 2 * size_t(s) * s;
  int* kept1 = B.kept.p;
  int* kept2 = kept1 + s;
  {
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(opted.load() & bit)) {
      MTF_CUDA(cudaFuncSetAttribute(k_bchol, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 16));
      opted.fetch_or(bit);
    }
  }
  const size_t chol_smem = 2 * size_t(s) * s * sizeof(double2);
  // pinned slot layout (doubles): H1 (m+1) s s complex | H2 | R1 | R2; kept flags and error word separately
  const size_t slot_h = 2 * size_t(m + 1) * s * s;
  const size_t slot_len = 2 * slot_h + 4 * size_t(s) * s + 2 * size_t(s) + 1;
  auto slot = [&](int J) { return B.pin + size_t(J & 1) * slot_len; };
  auto launch_step = [&](int J) {
    const int vb = J + vshift;
    float* Vj = B.V.p + 2 * int64_t(vb) * vstride;
    float* Zj = B.Z.p + 2 * int64_t(J) * vstride;
    if (pre) {
      launch_osrc_apply_f32(sys, Vj, ldn, Zj, ldn, s, st);
    } else {
      MTF_CUDA(cudaMemcpyAsync(Zj, Vj, size_t(s) * ldn * 8, cudaMemcpyDeviceToDevice, st));
    }
    launch_matvec_f32(sys, Zj, ldn, B.W.p, ldn, s, st);
    const int nq = (vb + 1) * s;
    MTF_CUDA(cudaMemsetAsync(Gpre, 0, 2 * size_t(s) * s * sizeof(double), st));
    MTF_CUDA(cudaMemsetAsync(G, 0, 2 * size_t(s) * s * sizeof(double), st));
    bdots(sys, B.W.p, s, ldn, B.W.p, ldn, s, ldn, Gpre, s, st);
    project(nq);
    bdots(sys, B.W.p, s, ldn, B.W.p, ldn, s, ldn, G, s, st);
    MTF_LAUNCH(KID_BCHOL, st, k_bchol<<<1, 256, chol_smem, st>>>(G, Gpre, nullptr, tau, s, R1, kept1));
    btrsm(B.W.p, ldn, R1, kept1, s, B.D.p, ldn, ldn, st);
    // second pass (CholQR2): the first leaves V = W R^-1 orthonormal only
    // to about cond(W) times the FP32 rounding; V_next = V R2^-1, R = R2 R1
    MTF_CUDA(cudaMemsetAsync(G, 0, 2 * size_t(s) * s * sizeof(double), st));
    bdots(sys, B.D.p, s, ldn, B.D.p, ldn, s, ldn, G, s, st);
    MTF_LAUNCH(KID_BCHOL, st, k_bchol<<<1, 256, chol_smem, st>>>(G, nullptr, kept1, 1e-3, s, R2, kept2));
    float* Vn = B.V.p + 2 * int64_t(vb + 1) * vstride;
    btrsm(B.D.p, ldn, R2, kept2, s, Vn, ldn, ldn, st);
    if (tc) tca_store(*B.tca, Vn, (vb + 1) * s, st);
    double* sl = slot(J);
    MTF_CUDA(cudaMemcpyAsync(sl, H1, 2 * size_t(nq) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(sl + slot_h, H2, 2 * size_t(nq) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(sl + 2 * slot_h, R1, 2 * size_t(s) * s * sizeof(double), cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(sl + 2 * slot_h + 2 * size_t(s) * s, R2, 2 * size_t(s) * s * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(B.kept_host + size_t(J & 1) * (2 * s + 1), kept1, 2 * size_t(s) * sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaMemcpyAsync(B.kept_host + size_t(J & 1) * (2 * s + 1) + 2 * s, err_word, sizeof(int),
                             cudaMemcpyDeviceToHost, st));
    MTF_CUDA(cudaEventRecord(B.ev[J & 1], st));
  };

  std::vector<cdouble> h, Rr1(size_t(s) * s), Rr2(size_t(s) * s), Rn(size_t(s) * s);
  int steps = 0;
  mtf_status status = MTF_OK;
  if (!reached && grow && J0 < Jend) {
    launch_step(J0);
    for (int J = J0; J < Jend; ++J) {
      if (J + 1 < Jend) launch_step(J + 1);
      MTF_CUDA(cudaEventSynchronize(B.ev[J & 1]));
      const double* sl = slot(J);
      const int* kh = B.kept_host + size_t(J & 1) * (2 * s + 1);
      if (kh[2 * s] != 0) {
        status = MTF_ERR_TIMEOUT;
        break;
      }
      const int nq = (J + vshift + 1) * s;
      h.assign(size_t(nq) * s, cdouble(0));
      bool finite = true;
      for (int q = 0; q < nq; ++q)
        for (int c = 0; c < s; ++c) {
          const size_t o = 2 * (size_t(q) * s + c);
          const cdouble v(sl[o] + sl[slot_h + o], sl[o + 1] + sl[slot_h + o + 1]);
          finite = finite && std::isfinite(v.real()) && std::isfinite(v.imag());
          h[size_t(c) * nq + q] = v;
        }
      const double* r1 = sl + 2 * slot_h;
      const double* r2 = r1 + 2 * size_t(s) * s;
      for (size_t t = 0; t < size_t(s) * s; ++t) {
        Rr1[t] = cdouble(r1[2 * t], r1[2 * t + 1]);
        Rr2[t] = cdouble(r2[2 * t], r2[2 * t + 1]);
      }
      if (!finite) {
        status = MTF_ERR_NAN;
        break;
      }
      for (int c = 0; c < s; ++c)
        for (int i = 0; i < s; ++i) {
          cdouble a = 0;
          if (i <= c)
            for (int p = i; p <= c; ++p) a += Rr2[size_t(p) * s + i] * Rr1[size_t(c) * s + p];
          Rn[size_t(c) * s + i] = a;
        }
      if (!lsq.add_block(h.data(), nq / s, Rn.data(), est.data())) break;
      ++steps;
      int nk = 0;
      for (int c = 0; c < s; ++c) nk += kh[c];
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
      if (nk == 0) break;  // the space is exhausted: the next cycle starts from the new residual
    }
    MTF_CUDA(cudaStreamSynchronize(st));  // a step queued past the last one has finished
  }
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
  B.rec_ok = true;
  return MTF_OK;
}

}  // namespace mtf
