// Real FP32 matrix products on the fifth-generation tensor cores for the
// learned correction's network (forward, backward and weight gradients):
//   D(r, c) op= sum_k A(r, k) B(c, k),   r < M, c < N, k < K,
// with A, B and D given by element strides, so that feature-major and
// row-major operands are read in place.  Each operand is scaled by a power
// of two (its largest entry below 2^14) and split into FP16 hi + lo tiles
// (the split of tc_plan.h: hi*hi + hi*lo + lo*hi, FP32 sums, about 2^-22
// relative); an operand may carry an implicit row or column of ones (the
// bias of an augmented [W | b] layer).  Work units (row tile of 128, column
// tile of NB <= 128, a range of 64-wide K chunks) run on k_tc_stream<2, NB,
// 0> (tc_stream.cuh); their raw sums are added in a fixed order, unscaled and
// passed through the epilogue op by k_tg_reduce.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "common.h"
#include "tc.cuh"
#include "tc_gemm.h"
#include "tc_plan.h"
#include "tc_stream.cuh"

namespace mtf {

void tc_encode_map(void* map, const void* base, int rows, int parts, int64_t count);

struct TcGemm {
  DevBuf<__half> A, B;
  DevBuf<float> part;
  DevBuf<int4> units;
  DevBuf<unsigned> amax;  // largest |A|, |B| (float bits)
  CUtensorMap amap{}, bmap{};
  const void* amap_ptr = nullptr;
  const void* bmap_ptr = nullptr;
  int64_t amap_n = 0, bmap_n = 0;
  int bmap_nb = 0;
  int n_cta = 0;
};

TcGemm* tg_create() { return new TcGemm(); }
void tg_destroy(TcGemm* g) { delete g; }

// largest |X(r, k)| over r < R, k < Kv (strided) into *out (float bits, atomicMax)
__global__ void k_tg_amax(const float* __restrict__ X, int64_t sr, int64_t sk, int64_t R, int64_t Kv, float init,
                          unsigned* __restrict__ out) {
  float m = init;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < R * Kv; t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = sr == 1 ? t % R : t / Kv, k = sr == 1 ? t / R : t % Kv;
    m = fmaxf(m, fabsf(X[r * sr + k * sk]));
  }
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__device__ __forceinline__ float tg_scale(unsigned bits) {
  const float a = __uint_as_float(bits);
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, 14 - ex);
}

// tiles of rows_per_tile rows x 64 K-values, parts hi / lo, tile (t_r, t_k)
// at index t_r * n_kc + t_k; value (r, k) = X(r, k) for r < Rv, k < Kv, 1 on
// the ones row (r == ones_r, k < Kv) or ones column (k == ones_k, r < Rv),
// else 0.  Thread = (tile, row, group of 8 K-values).
__global__ void k_tg_pack(const float* __restrict__ X, int64_t sr, int64_t sk, int64_t Rv, int64_t Kv, int ones_r,
                          int ones_k, int rows_per_tile, int64_t n_rt, int64_t n_kc, const unsigned* __restrict__ amax,
                          __half* __restrict__ T) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_rt * n_kc * rows_per_tile * 8) return;
  const int g = int(t % 8);
  const int row = int((t / 8) % rows_per_tile);
  const int64_t tile = t / (8 * int64_t(rows_per_tile));
  const int64_t tr = tile / n_kc, tk = tile % n_kc;
  const int64_t r = tr * rows_per_tile + row;
  const float sc = tg_scale(*amax);
  __align__(16) __half hi[8], lo[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t k = tk * 64 + 8 * g + e;
    float v = 0.f;
    if (r < Rv && k < Kv) v = X[r * sr + k * sk];
    else if ((r == ones_r && k < Kv) || (k == ones_k && r < Rv)) v = 1.f;
    v *= sc;
    hi[e] = __float2half_rn(v);
    lo[e] = __float2half_rn(v - __half2float(hi[e]));
  }
  const int64_t base = ((tile * 2) * rows_per_tile + row) * 64 + 8 * g;
  *reinterpret_cast<uint4*>(T + base) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(T + base + int64_t(rows_per_tile) * 64) = *reinterpret_cast<const uint4*>(lo);
}

// D(r, c) for r < M, c < N: the sum of the P pieces of unit (mt, nt) in order,
// unscaled, through op (0 store, 1 ReLU, 2 keep where mask(r, c) > 0, 3 add)
__global__ void k_tg_reduce(const float* __restrict__ part, int nb, int NT, int P, int64_t M, int64_t N,
                            const unsigned* __restrict__ amax, int op, const float* __restrict__ mask, int64_t mr,
                            int64_t mc, float* __restrict__ D, int64_t dr, int64_t dc) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= M * N) return;
  // consecutive threads take consecutive entries along the unit-stride side of D
  const int64_t r = dr == 1 ? t % M : t / N, c = dr == 1 ? t / M : t % N;
  const int64_t mt = r / kTcRows, row = r % kTcRows, nt = c / nb, col = c % nb;
  float v = 0.f;
  for (int p = 0; p < P; ++p) v += part[(((mt * NT + nt) * P + p) * kTcRows + row) * nb + col];
  v /= tg_scale(amax[0]) * tg_scale(amax[1]);
  float* d = D + r * dr + c * dc;
  if (op == 1) v = fmaxf(v, 0.f);
  if (op == 2) v = mask[r * mr + c * mc] > 0.f ? v : 0.f;
  if (op == 3) v += *d;
  *d = v;
}

template <int NB>
static void tg_run(TcGemm& g, const TgOperand& A, const TgOperand& B, int64_t M, int64_t N, int64_t K,
                   const TgOut& out, cudaStream_t s) {
  const int64_t n_mt = (M + kTcRows - 1) / kTcRows, n_nt = (N + NB - 1) / NB, n_kc = (K + 63) / 64;
  // K pieces: enough units to fill the SMs, at least 4 chunks each, at most 32 pieces
  int P = int(std::max<int64_t>(1, std::min<int64_t>({n_kc / 4, 32, (2 * int64_t(g.n_cta) + n_mt * n_nt - 1) /
                                                                         (n_mt * n_nt)})));
  const int64_t L = (n_kc + P - 1) / P;
  P = int((n_kc + L - 1) / L);
  const size_t na = size_t(n_mt * n_kc) * 2 * kTcRows * 64, nbh = size_t(n_nt * n_kc) * 2 * NB * 64;
  if (g.A.n < na) g.A.alloc(na);
  if (g.B.n < nbh) g.B.alloc(nbh);
  const size_t np = size_t(n_mt * n_nt * P) * kTcRows * NB;
  if (g.part.n < np) g.part.alloc(np);
  if (g.amap_ptr != g.A.p || g.amap_n < n_mt * n_kc) {
    g.amap_n = int64_t(g.A.n / (2 * kTcRows * 64));
    tc_encode_map(&g.amap, g.A.p, kTcRows, 2, g.amap_n);
    g.amap_ptr = g.A.p;
  }
  if (g.bmap_ptr != g.B.p || g.bmap_nb != NB || g.bmap_n < n_nt * n_kc) {
    g.bmap_n = int64_t(g.B.n / (2 * NB * 64));
    tc_encode_map(&g.bmap, g.B.p, NB, 2, g.bmap_n);
    g.bmap_ptr = g.B.p;
    g.bmap_nb = NB;
  }
  // operand scales, packed tiles
  MTF_CUDA(cudaMemsetAsync(g.amax.p, 0, 2 * sizeof(unsigned), s));
  // the ones of a bias row or column count as entries of their operand
  const float oa = (A.ones_r >= 0 || A.ones_k >= 0) ? 1.f : 0.f, ob = (B.ones_r >= 0 || B.ones_k >= 0) ? 1.f : 0.f;
  MTF_LAUNCH(KID_MLP, s, k_tg_amax<<<256, 256, 0, s>>>(A.X, A.sr, A.sk, A.Rv, A.Kv, oa, g.amax.p));
  MTF_LAUNCH(KID_MLP, s, k_tg_amax<<<256, 256, 0, s>>>(B.X, B.sr, B.sk, B.Rv, B.Kv, ob, g.amax.p + 1));
  const int64_t ta = n_mt * n_kc * kTcRows * 8, tb = n_nt * n_kc * NB * 8;
  MTF_LAUNCH(KID_MLP, s, k_tg_pack<<<unsigned((ta + 255) / 256), 256, 0, s>>>(
      A.X, A.sr, A.sk, A.Rv, A.Kv, A.ones_r, A.ones_k, kTcRows, n_mt, n_kc, g.amax.p, g.A.p));
  MTF_LAUNCH(KID_MLP, s, k_tg_pack<<<unsigned((tb + 255) / 256), 256, 0, s>>>(
      B.X, B.sr, B.sk, B.Rv, B.Kv, B.ones_r, B.ones_k, NB, n_nt, n_kc, g.amax.p + 1, g.B.p));
  // units in (mt, nt, piece) order
  std::vector<int4> un;
  un.reserve(size_t(n_mt * n_nt * P));
  for (int64_t mt = 0; mt < n_mt; ++mt)
    for (int64_t nt = 0; nt < n_nt; ++nt)
      for (int p = 0; p < P; ++p) {
        const int64_t k0 = int64_t(p) * L, k1 = std::min<int64_t>(n_kc, k0 + L);
        un.push_back(make_int4(int(mt * n_kc), int(nt * n_kc), int(k0), int(k1)));
      }
  if (g.units.n < un.size()) g.units.alloc(un.size());
  MTF_CUDA(cudaMemcpyAsync(g.units.p, un.data(), un.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  using Cfg = TcsCfg<2, NB>;
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_tc_stream<2, NB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem)));
    opted.fetch_or(bit);
  }
  TcUnits units;
  units.list = g.units.p;
  const int nu = int(un.size());
  MTF_LAUNCH(KID_MLP, s, k_tc_stream<2, NB, 0><<<unsigned(std::min(nu, g.n_cta)), 192, Cfg::smem, s>>>(
      g.amap, g.bmap, units, nu, nullptr, nullptr, g.part.p, nullptr, 0, 0, 0, nullptr, out.err, TcTtOut{}));
  MTF_LAUNCH(KID_MLP, s, k_tg_reduce<<<unsigned((M * N + 255) / 256), 256, 0, s>>>(
      g.part.p, NB, int(n_nt), P, M, N, g.amax.p, out.op, out.mask, out.mr, out.mc, out.D, out.dr, out.dc));
  // the unit list is host memory of this call
  MTF_CUDA(cudaStreamSynchronize(s));
}

void tc_gemm(TcGemm& g, const TgOperand& A, const TgOperand& B, int64_t M, int64_t N, int64_t K, const TgOut& out,
             cudaStream_t s) {
  MTF_REQUIRE(M >= 1 && N >= 1 && K >= 1, MTF_ERR_ARG, "tc_gemm: empty product");
  if (!g.amax.p) g.amax.alloc(2);
  if (g.n_cta == 0) {
    int dev = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    MTF_CUDA(cudaDeviceGetAttribute(&g.n_cta, cudaDevAttrMultiProcessorCount, dev));
  }
  // column tiles of at most 128; narrow products take the narrowest kernel
  if (N <= 16) tg_run<16>(g, A, B, M, N, K, out, s);
  else if (N <= 32) tg_run<32>(g, A, B, M, N, K, out, s);
  else if (N <= 64) tg_run<64>(g, A, B, M, N, K, out, s);
  else tg_run<128>(g, A, B, M, N, K, out, s);
}

}  // namespace mtf
