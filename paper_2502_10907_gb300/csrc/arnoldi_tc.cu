// Block Gram-Schmidt projections of the block FGMRES cycle on the tensor
// cores: H = V^H W and W -= V H for the s vectors of W against the nq basis
// vectors of V, with FP16 hi + lo operands and FP32 accumulation in TMEM
// (the formulation of the tensor-core matvec, tc_plan.h).
//
// The basis is kept in two tiled FP16 hi / lo copies (entries scaled by 2^14;
// basis vectors have unit norm) so that both products read K-major tiles:
//  - dots copy: tile (g, kc) = basis vectors 128 g .. 128 g + 127 x entries
//    32 kc .. 32 kc + 31, rows = vectors, (re, im) interleaved along K = the
//    entry index: H[q, c] = sum_k conj(v_q[k]) w_c[k] with input columns
//    (w_re, w_im) and (w_im, -w_re) per complex w_c;
//  - update copy: tile (e, b) = entries 128 e .. 128 e + 127 x basis vectors
//    32 b .. 32 b + 31, rows = entries, (re, im) interleaved along K = the
//    basis index: (V H)[k, c] with input columns (H_re, -H_im) and
//    (H_im, H_re) per complex H[:, c].
// The dots may read the hi parts of the basis alone (two products, half the
// basis bytes): a basis entry then enters the dots rounded to FP16.  Classical
// Gram-Schmidt twice tolerates that error in its coefficients (the second
// pass measures what the first left, and the rounding errors of the basis
// entries do not correlate with W), while the update W -= V H, which carries
// the Arnoldi relation M Z = V H, keeps hi + lo.
// Dots units (basis group g, a range of entry chunks) write row sums that a
// reduction adds in FP64 into H; update units (entry group e, all basis
// chunks) subtract their product from W directly.  Both unit sets follow a
// rule the kernel evaluates (no host lists), so the steps of the block cycle
// can be queued ahead of the host.  The stream kernel is the
// matvec's pipeline (TMA producer, one MMA-issuing thread, four epilogue
// warps, two TMEM buffers) with one operator of two parts.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "common.h"
#include "tc.cuh"
#include "tc_plan.h"
#include "tc_stream.cuh"

namespace mtf {

// tensor-map encoder and helpers of the tensor-core matvec (mv_tc.cu)
void tc_encode_map(void* map, const void* base, int rows, int parts, int64_t count);
void tc_encode_map_first(void* map, const void* base, int rows, int parts, int64_t count);

constexpr float kBasisScale = 16384.f;  // 2^14: unit-norm basis entries stay below the FP16 range limit

__device__ __forceinline__ float tca_scale(unsigned bits) {
  const float a = __uint_as_float(bits);
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, 14 - ex);
}
__device__ __forceinline__ float tca_inv_scale(unsigned bits) {
  const float a = __uint_as_float(bits);
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, ex - 14);
}
__device__ __forceinline__ void tca_split(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// new basis vectors q0 .. q0 + s - 1 (FP32, stride ldn) into the dots copy:
// thread = (vector, group of 4 entries), entries fastest
__global__ void k_tca_store_dots(const float* __restrict__ Vn, int64_t ldn, int q0, int s, int nkc,
                                 __half* __restrict__ Vd) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t ng = ldn / 4;
  if (t >= ng * s) return;
  const int q = int(t / ng);
  const int64_t k = (t % ng) * 4;
  const int qq = q0 + q;
  const float4* src = reinterpret_cast<const float4*>(Vn + 2 * (int64_t(q) * ldn + k));
  const float4 a = src[0], b = src[1];
  const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  __half hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) tca_split(v[i] * kBasisScale, hi[i], lo[i]);
  *reinterpret_cast<uint4*>(Vd + tca_dots_half(qq, k, nkc, 0)) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(Vd + tca_dots_half(qq, k, nkc, 1)) = *reinterpret_cast<const uint4*>(lo);
}

// the same vectors into the update copy: thread = (entry, vector), vectors fastest
__global__ void k_tca_store_upd(const float* __restrict__ Vn, int64_t ldn, int q0, int s, int nbc,
                                __half* __restrict__ Vu) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= ldn * s) return;
  const int q = int(t % s);
  const int64_t k = t / s;
  const int qq = q0 + q;
  const float2 v = reinterpret_cast<const float2*>(Vn + 2 * int64_t(q) * ldn)[k];
  __half h[2], l[2];
  tca_split(v.x * kBasisScale, h[0], l[0]);
  tca_split(v.y * kBasisScale, h[1], l[1]);
  *reinterpret_cast<__half2*>(Vu + tca_upd_half(qq, k, nbc, 0)) = *reinterpret_cast<const __half2*>(h);
  *reinterpret_cast<__half2*>(Vu + tca_upd_half(qq, k, nbc, 1)) = *reinterpret_cast<const __half2*>(l);
}

// colmax[c] = max |re|, |im| of FP32 column c (n complex entries, stride ld)
__global__ void k_tca_colmax32(const float* __restrict__ W, int64_t ld, int64_t n, unsigned* __restrict__ colmax) {
  const int c = blockIdx.y;
  const float2* w = reinterpret_cast<const float2*>(W + 2 * int64_t(c) * ld);
  float m = 0.f;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const float2 v = w[k];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(colmax + c, __float_as_uint(m));
}

// colmax[c] = max over q < nq of |re|, |im| of H[q, c] (FP64, leading dim ldh)
__global__ void k_tca_colmax64(const double* __restrict__ H, int nq, int ldh, unsigned* __restrict__ colmax) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int c = blockIdx.y;
  float m = 0.f;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
    const double* h = H + 2 * (int64_t(q) * ldh + c);
    m = fmaxf(m, fmaxf(fabsf(float(h[0])), fabsf(float(h[1]))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(colmax + c, __float_as_uint(m));
}

// dots input chunks from W: column 2 c + f, form 0 (w_re, w_im), form 1
// (w_im, -w_re); thread = (chunk, column, group of 4 entries)
__global__ void k_tca_w_to_b(const float* __restrict__ W, int64_t ldw, int s, int nkc, int nb,
                             const unsigned* __restrict__ colmax, __half* __restrict__ Bd) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(nkc) * nb * 8) return;
  const int64_t kc = t / (int64_t(nb) * 8);
  const int col = int((t / 8) % nb), g = int(t % 8);
  const int c = col >> 1, form = col & 1;
  __half hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) hi[i] = lo[i] = __float2half_rn(0.f);
  if (c < s) {
    const float sc = tca_scale(colmax[c]);
    const float2* w = reinterpret_cast<const float2*>(W + 2 * int64_t(c) * ldw) + kc * kTcCols + 4 * g;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 v = w[i];
      const float a = form == 0 ? v.x : v.y, b = form == 0 ? v.y : -v.x;
      tca_split(a * sc, hi[2 * i], lo[2 * i]);
      tca_split(b * sc, hi[2 * i + 1], lo[2 * i + 1]);
    }
  }
  *reinterpret_cast<uint4*>(Bd + tc_b_index(kc, 0, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(Bd + tc_b_index(kc, 1, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(lo);
}

// update input chunks from H (FP64, q < nq, leading dim ldh): column 2 c + f,
// form 0 (H_re, -H_im), form 1 (H_im, H_re); thread = (chunk, column, group
// of 4 vectors)
__global__ void k_tca_h_to_b(const double* __restrict__ H, int nq, int s, int ldh, int nbc, int nb,
                             const unsigned* __restrict__ colmax, __half* __restrict__ Bu) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(nbc) * nb * 8) return;
  const int b = int(t / (int64_t(nb) * 8));
  const int col = int((t / 8) % nb), g = int(t % 8);
  const int c = col >> 1, form = col & 1;
  __half hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) hi[i] = lo[i] = __float2half_rn(0.f);
  if (c < s) {
    const float sc = tca_scale(colmax[c]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = b * 32 + 4 * g + i;
      if (q < nq) {
        const double* h = H + 2 * (int64_t(q) * ldh + c);
        const float re = float(h[0]), im = float(h[1]);
        const float x = form == 0 ? re : im, y = form == 0 ? -im : re;
        tca_split(x * sc, hi[2 * i], lo[2 * i]);
        tca_split(y * sc, hi[2 * i + 1], lo[2 * i + 1]);
      }
    }
  }
  *reinterpret_cast<uint4*>(Bu + tc_b_index(b, 0, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(Bu + tc_b_index(b, 1, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(lo);
}

// H[q, c] (at H + 2 (q ldh + c)) = (sum over the P pieces of basis group
// q / 128 of the raw sums) x the inverse scales, in FP64; thread = (q, c)
__global__ void k_tca_dots_reduce(const float* __restrict__ part, int nb, int P, int nq, int s,
                                  const unsigned* __restrict__ colmax, double* __restrict__ H, int ldh) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(nq) * s) return;
  const int q = int(t / s), c = int(t % s);
  const int g = q / kTcRows, row = q % kTcRows;
  // FP32 partials added in double-float (two-sum: Knuth's error-free
  // transformation) on the FP32 pipes, rounded to FP64 once
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (int p = 0; p < P; ++p) {
    const float2 v = *reinterpret_cast<const float2*>(part + (size_t(g * P + p) * kTcRows + row) * nb + 2 * c);
    float s1 = rh + v.x, bb = s1 - rh;
    rl += (rh - (s1 - bb)) + (v.x - bb);
    rh = s1;
    s1 = ih + v.y;
    bb = s1 - ih;
    il += (ih - (s1 - bb)) + (v.y - bb);
    ih = s1;
  }
  const double re = double(rh) + double(rl), im = double(ih) + double(il);
  const double sc = double(tca_inv_scale(colmax[c])) / double(kBasisScale);
  const int64_t o = 2 * (int64_t(q) * ldh + c);
  H[o] = re * sc;
  H[o + 1] = im * sc;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr int kTcaMaxCols = 64;  // columns of one projection pass (NB = 128)

struct TcArnoldi {
  int s = 0, m = 0;
  int64_t ldn = 0;
  int G = 0, nkc = 0, E = 0, nbc = 0;  // basis groups, entry chunks, entry groups, basis chunks
  DevBuf<__half> Vd, Vu, Bd, Bu;
  DevBuf<float> part;
  DevBuf<unsigned> cm;                 // colmax of W (s) and of H (s)
  size_t h_cap = 0;                    // units the partial buffer holds
  int n_cta = 0, b_nb = 0;
  CUtensorMap vd_map{}, vu_map{}, bd_map{}, bu_map{};
  CUtensorMap vd_hi_map{};             // the dots copy's FP16 hi parts alone
  bool dots_hi = false;                // dots from the basis's hi part (two products)

};

TcArnoldi* tca_create() { return new TcArnoldi(); }
void tca_destroy(TcArnoldi* t) { delete t; }
void tca_set_dots_hi(TcArnoldi& t, bool on) { t.dots_hi = on; }

static int tca_nb(int nc) { return 2 * nc <= 16 ? 16 : 2 * nc <= 32 ? 32 : 2 * nc <= 64 ? 64 : 128; }

void tca_prepare(TcArnoldi& t, int s, int m, int64_t ldn, cudaStream_t st) {
  MTF_REQUIRE(s >= 1 && s <= 64 && ldn % 64 == 0, MTF_ERR_ARG, "tensor-core Arnoldi: 1..64 columns, padded length");
  if (t.s == s && t.m == m && t.ldn == ldn) return;
  t.s = s;
  t.m = m;
  t.ldn = ldn;
  const int64_t nvec = int64_t(m + 1) * s;
  t.G = int((nvec + kTcRows - 1) / kTcRows);
  t.nkc = int(ldn / kTcCols);
  t.E = int((ldn + kTcRows - 1) / kTcRows);
  t.nbc = int((nvec + 31) / 32);
  t.Vd.alloc(size_t(tca_dots_halves(nvec, ldn)));
  t.Vu.alloc(size_t(tca_upd_halves(nvec, ldn)));
  MTF_CUDA(cudaMemsetAsync(t.Vd.p, 0, t.Vd.n * sizeof(__half), st));
  MTF_CUDA(cudaMemsetAsync(t.Vu.p, 0, t.Vu.n * sizeof(__half), st));
  t.Bd.alloc(size_t(t.nkc) * 2 * 128 * 64);
  t.Bu.alloc(size_t(t.nbc) * 2 * 128 * 64);
  t.cm.alloc(size_t(2) * kTcaMaxCols);
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  MTF_CUDA(cudaDeviceGetAttribute(&t.n_cta, cudaDevAttrMultiProcessorCount, dev));
  // dots units: up to 4 per CTA over the basis groups in use; update units: one per entry group
  const size_t cap = size_t(4 * t.n_cta + t.G) + 16;
  t.part.alloc(cap * kTcRows * 128);
  t.h_cap = cap;
  tc_encode_map(&t.vd_map, t.Vd.p, kTcRows, 2, int64_t(t.G) * t.nkc);
  tc_encode_map_first(&t.vd_hi_map, t.Vd.p, kTcRows, 2, int64_t(t.G) * t.nkc);
  tc_encode_map(&t.vu_map, t.Vu.p, kTcRows, 2, int64_t(t.E) * t.nbc);
  t.b_nb = 0;
}

// B maps for width nb (the chunk buffers hold the widest)
static void tca_bmaps(TcArnoldi& t, int nb) {
  if (t.b_nb == nb) return;
  tc_encode_map(&t.bd_map, t.Bd.p, nb, 2, t.nkc);
  tc_encode_map(&t.bu_map, t.Bu.p, nb, 2, t.nbc);
  t.b_nb = nb;
}

// basis vectors q0 .. q0 + s - 1 (FP32 columns of stride ldn) into both copies
void tca_store(TcArnoldi& t, const float* Vn, int q0, cudaStream_t st) {
  const int64_t n1 = t.ldn / 4 * t.s, n2 = t.ldn * t.s;
  MTF_LAUNCH(KID_BSTORE, st, launch_pdl(k_tca_store_dots, dim3(unsigned((n1 + 255) / 256)), dim3(256), 0, st,
      Vn, t.ldn, q0, t.s, t.nkc,
                                                                                        t.Vd.p));
  MTF_LAUNCH(KID_BSTORE, st, launch_pdl(k_tca_store_upd, dim3(unsigned((n2 + 255) / 256)), dim3(256), 0, st,
      Vn, t.ldn, q0, t.s, t.nbc,
                                                                                       t.Vu.p));
}

template <int NPA, int NB, int EPI>
static void tca_launch(TcArnoldi& t, const CUtensorMap& amap, const CUtensorMap& bmap, const TcUnits& units,
                       int n_units, float* W, int nc, int64_t n_limit, const unsigned* cm, unsigned* err, int kid,
                       cudaStream_t st) {
  using Cfg = TcsCfg<NPA, NB>;
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_tc_stream<NPA, NB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(Cfg::smem)));
    opted.fetch_or(bit);
  }
  const unsigned grid = unsigned(std::min(n_units, t.n_cta));
  MTF_LAUNCH(kid, st, k_tc_stream<NPA, NB, EPI><<<grid, 192, Cfg::smem, st>>>(amap, bmap, units, n_units, nullptr,
                                                                              nullptr, t.part.p, W, t.ldn, nc, n_limit,
                                                                              cm, err, TcTtOut{}));
}

template <int NB>
static void tca_project_nb(TcArnoldi& t, int nq, float* W, int nc, double* H, int ldh, unsigned* err, cudaStream_t st) {
  tca_bmaps(t, NB);
  unsigned* cmw = t.cm.p;
  unsigned* cmh = t.cm.p + kTcaMaxCols;
  MTF_CUDA(cudaMemsetAsync(t.cm.p, 0, size_t(2) * kTcaMaxCols * sizeof(unsigned), st));
  // H = V^H W: units (basis group g, a piece of the entry chunks)
  MTF_LAUNCH(KID_TCA_PREP, st, k_tca_colmax32<<<dim3(64, unsigned(nc)), 256, 0, st>>>(W, t.ldn, t.ldn, cmw));
  const int64_t nthr = int64_t(t.nkc) * NB * 8;
  MTF_LAUNCH(KID_TCA_PREP, st, launch_pdl(k_tca_w_to_b, dim3(unsigned((nthr + 255) / 256)), dim3(256), 0, st,
      W, t.ldn, nc, t.nkc, NB, cmw,
                                                                                      t.Bd.p));
  const int g_used = (nq + kTcRows - 1) / kTcRows;
  const int P = std::max(1, std::min({t.nkc, 32, (4 * t.n_cta + g_used - 1) / g_used}));
  const int L = (t.nkc + P - 1) / P;
  const int Pn = (t.nkc + L - 1) / L;
  const int nu = g_used * Pn;
  MTF_REQUIRE(size_t(nu) <= t.h_cap, MTF_ERR_ARG, "tensor-core Arnoldi: too many units for the partial buffer");
  TcUnits ud;
  ud.kind = 1;
  ud.a = t.nkc;
  ud.b = L;
  ud.c = Pn;
  if (t.dots_hi) {
    prof_bytes(KID_DOTS, (double(nq) * 4.0 + double(nc) * 8.0) * double(t.ldn));
    tca_launch<1, NB, 0>(t, t.vd_hi_map, t.bd_map, ud, nu, nullptr, nc, 0, cmw, err, KID_DOTS, st);
  } else {
    prof_bytes(KID_DOTS, double(nq + nc) * double(t.ldn) * 8.0);
    tca_launch<2, NB, 0>(t, t.vd_map, t.bd_map, ud, nu, nullptr, nc, 0, cmw, err, KID_DOTS, st);
  }
  const unsigned gr = unsigned((int64_t(nq) * nc + 255) / 256);
  MTF_LAUNCH(KID_TCA_PREP, st, launch_pdl(k_tca_dots_reduce, dim3(gr), dim3(256), 0, st,
      t.part.p, NB, Pn, nq, nc, cmw, H, ldh));
  // W -= V H: one unit per entry group, over the basis chunks in use
  MTF_LAUNCH(KID_TCA_PREP, st, launch_pdl(k_tca_colmax64, dim3(8, unsigned(nc)), dim3(256), 0, st,
      H, nq, ldh, cmh));
  const int nbc_used = (nq + 31) / 32;
  const int64_t nthu = int64_t(nbc_used) * NB * 8;
  MTF_LAUNCH(KID_TCA_PREP, st, launch_pdl(k_tca_h_to_b, dim3(unsigned((nthu + 255) / 256)), dim3(256), 0, st,
      H, nq, nc, ldh, nbc_used, NB,
                                                                                      cmh, t.Bu.p));
  TcUnits uu;
  uu.kind = 2;
  uu.a = t.nbc;
  uu.b = nbc_used;
  prof_bytes(KID_AXPY, double(nq + 2 * nc) * double(t.ldn) * 8.0);
  tca_launch<2, NB, 1>(t, t.vu_map, t.bu_map, uu, t.E, W, nc, t.ldn, cmh, err, KID_AXPY, st);
}

// H[q, c] (q < nq, c < nc; complex FP64 at H + 2 (q ldh + c)) = V^H W, then
// W -= V H, for the first nq basis vectors stored by tca_store and the nc
// columns of W (stride ldn), in passes of up to 64 columns
void tca_project(TcArnoldi& t, int nq, float* W, int nc, double* H, int ldh, unsigned* err, cudaStream_t st) {
  MTF_REQUIRE(nq >= 1 && int64_t(nq) <= int64_t(t.m + 1) * t.s && nc >= 1, MTF_ERR_ARG,
              "tensor-core Arnoldi: basis size");
  for (int c0 = 0; c0 < nc; c0 += kTcaMaxCols) {
    const int w = std::min(kTcaMaxCols, nc - c0);
    float* Wg = W + 2 * int64_t(c0) * t.ldn;
    double* Hg = H + 2 * c0;
    const int nb = tca_nb(w);
    if (nb == 16) tca_project_nb<16>(t, nq, Wg, w, Hg, ldh, err, st);
    else if (nb == 32) tca_project_nb<32>(t, nq, Wg, w, Hg, ldh, err, st);
    else if (nb == 64) tca_project_nb<64>(t, nq, Wg, w, Hg, ldh, err, st);
    else tca_project_nb<128>(t, nq, Wg, w, Hg, ldh, err, st);
  }
}

}  // namespace mtf
