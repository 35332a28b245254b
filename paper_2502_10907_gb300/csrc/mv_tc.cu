// Block matvec of the mixed inner solver on the fifth-generation tensor cores
// (Eq. 16 applied as y = 2 A x + X x, block by block): every stored entry of
// the dense {T_i, K_i} is read ONCE per apply for up to 32 right-hand sides,
// instead of once per group of 4 in the FMA stream.
//
// Formulation and layout: tc_plan.h (interleaved complex rows, two real
// input columns per complex input, FP16 hi + lo split of both operands after
// power-of-two scaling, three products with FP32 accumulation).
//
// Kernel k_mv_tc (one persistent CTA per SM, 6 warps):
//  - warp 0, one lane: producer.  For every chunk of the CTA's units it
//    loads the 64 KB operator tile (4 parts) and the input chunk (hi, lo)
//    with two cp.async.bulk.tensor.4d copies (128-byte swizzle) into a ring
//    of S stages, completing on the stage's "full" mbarrier;
//  - warp 1: allocates TMEM (two accumulator buffers of 2 NB columns:
//    T products, K products); one lane issues per K = 16 step the six
//    tcgen05.mma of the split products and commits each stage back to its
//    "empty" barrier, and each finished unit to the buffer's "full" barrier;
//  - warps 2-5: epilogue.  Each reads its 32 TMEM lanes (rows) of the
//    finished buffer with tcgen05.ld and writes the unit's raw row sums to a
//    partial buffer, then frees the TMEM buffer.
// k_mv_tc_combine then adds the pieces of each row in order, undoes the
// scalings and applies 2 (K u_D + rho^-1 T u_N), 2 (-rho T u_D + K u_N) and
// the exchange rows, as the FMA stream's combine does.  Every wait is
// bounded (0.5 s) and ends in the error word.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "common.h"
#include "tc.cuh"
#include "tc_plan.h"
#include "tc_stream.cuh"

namespace mtf {

struct TcMatvec {
  TcPlan plan;
  int n_cta = 0;
  bool planned = false, built = false;
  // launch plan (the autotuner's choice; 0 = plan_tc's defaults, one CTA per SM)
  int waves = 0, min_len = 0, grid = 0;
  bool prefer_fma = false;             // wide applies on the FMA streams instead
  DevBuf<__half> A;                    // tiled hi / lo operator
  DevBuf<unsigned> amax;               // per block: largest |re|, |im| of T and K (float bits)
  DevBuf<int4> units, tile_info;       // unit {blk, mt, kc0, kc1}; tile {blk, mt, kc, 0}
  DevBuf<int2> chunk_info;             // chunk {blk, kc}
  DevBuf<int> sched, sched_off, blk_unit_base, blk_pieces, blk_nkc;
  DevBuf<int64_t> blk_tile_base, blk_chunk_base;
  DevBuf<__half> B;                    // input chunks for up to 32 right-hand sides
  DevBuf<float> part;                  // per unit: 128 rows x 2 NB raw sums
  DevBuf<unsigned> colmax;             // per right-hand side of a pass (float bits)
  CUtensorMap amap{}, bmap{};
  const void* amap_ptr = nullptr;
  const void* bmap_ptr = nullptr;
  int bmap_nb = 0;
  // block-OSRC on the tensor cores: the FP16 T~ in the same row tiles
  // (one part), units {a_base, b_base, kc0, kc1} of the same plan
  DevBuf<int4> units_ab;
  DevBuf<__half> Aos;
  DevBuf<int64_t> os_off, os_ld;       // per block: first entry and row stride of the FP16 T~
  CUtensorMap osmap{};
  const void* osmap_ptr = nullptr;
  bool os_built = false;
  // block-OSRC Type 2 (T~2 = i R, R real symmetric): R in FP16 row tiles of
  // 128 rows x 64 real columns (2 bytes per entry), real input chunks of 64
  // entries, units of its own plan (64 columns per chunk)
  struct Real {
    TcPlan plan;
    DevBuf<int4> units_ab, tile_info;
    DevBuf<int2> chunk_info;
    DevBuf<int> sched, sched_off, blk_unit_base, blk_pieces;
    DevBuf<__half> A, B;
    DevBuf<float> part;
    CUtensorMap amap{}, bmap{};
    const void* amap_ptr = nullptr;
    const void* bmap_ptr = nullptr;
    int bmap_nb = 0;
    bool planned = false;
  } osr;
};

void destroy_tc(TcMatvec* t) { delete t; }

// power-of-two scale s with amax * s < 2^14 (1 for amax = 0), and 1 / s
__device__ __forceinline__ float tc_scale(unsigned bits) {
  const float a = __uint_as_float(bits);
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, 14 - ex);
}
__device__ __forceinline__ float tc_inv_scale(unsigned bits) {
  const float a = __uint_as_float(bits);
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, ex - 14);
}

// hi = fp16(v), lo = fp16(v - hi)
__device__ __forceinline__ void tc_split(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// amax[i] = max over block i's stored T and K entries of |re|, |im|
__global__ void k_tc_blkmax(const float4* __restrict__ TK, const int64_t* __restrict__ blk_mat_off,
                            const int32_t* __restrict__ blk_N, unsigned* __restrict__ amax) {
  const int i = blockIdx.y;
  const int64_t N = blk_N[i];
  const float4* e = TK + blk_mat_off[i];
  float m = 0.f;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < N * N; t += int64_t(gridDim.x) * blockDim.x) {
    const float4 v = e[t];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax + i, __float_as_uint(m));
}

// Tiled hi / lo copy: thread = (tile, row, group g of 4 complex columns);
// writes 8 halves (16 bytes) into each of the 4 parts.
__global__ void __launch_bounds__(256) k_tc_tile_a(const float4* __restrict__ TK, const int4* __restrict__ tile_info,
                                                   const int64_t* __restrict__ blk_mat_off,
                                                   const int32_t* __restrict__ blk_N, const unsigned* __restrict__ amax,
                                                   int64_t n_tiles, __half* __restrict__ A) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_tiles * kTcRows * 8) return;
  const int64_t tile = t / (kTcRows * 8);
  const int row = int((t / 8) % kTcRows), g = int(t % 8);
  const int4 info = tile_info[tile];
  const int i = info.x, N = blk_N[i];
  const int r = info.y * kTcRows + row;
  const float s = tc_scale(amax[i]);
  __half h[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int n = info.z * kTcCols + 4 * g + q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < N && n < N) v = TK[blk_mat_off[i] + int64_t(r) * N + n];
    tc_split(v.x * s, h[0][2 * q], h[1][2 * q]);          // T re
    tc_split(v.y * s, h[0][2 * q + 1], h[1][2 * q + 1]);  // T im
    tc_split(v.z * s, h[2][2 * q], h[3][2 * q]);          // K re
    tc_split(v.w * s, h[2][2 * q + 1], h[3][2 * q + 1]);  // K im
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
    *reinterpret_cast<uint4*>(A + tc_a_index(tile, p, row, 8 * g)) = *reinterpret_cast<const uint4*>(h[p]);
}

// FP16 T~ tiles (one part): thread = (tile, row, group g of 4 complex
// columns); entries of block i at off[i] + r ld[i] + n as (re, im) halves
__global__ void __launch_bounds__(256) k_tc_tile_os(const __half2* __restrict__ T16, const int4* __restrict__ tile_info,
                                                    const int64_t* __restrict__ off, const int64_t* __restrict__ ld,
                                                    const int32_t* __restrict__ blk_N, int64_t n_tiles,
                                                    __half* __restrict__ A) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_tiles * kTcRows * 8) return;
  const int64_t tile = t / (kTcRows * 8);
  const int row = int((t / 8) % kTcRows), g = int(t % 8);
  const int4 info = tile_info[tile];
  const int i = info.x, N = blk_N[i];
  const int r = info.y * kTcRows + row;
  __half2 h[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int n = info.z * kTcCols + 4 * g + q;
    h[q] = (r < N && n < N) ? T16[off[i] + int64_t(r) * ld[i] + n] : __floats2half2_rn(0.f, 0.f);
  }
  *reinterpret_cast<uint4*>(A + tc_tile_index(tile, 1, 0, row, 8 * g)) = *reinterpret_cast<const uint4*>(h);
}

// FP16 tiles of R = Im T~ (block-OSRC Type 2, whose T~ = i R): thread =
// (tile, row, group g of 8 real columns); R(r, n) is the imaginary half of
// the FP16 copy's entry (r, n)
__global__ void __launch_bounds__(256) k_tc_tile_os_im(const __half2* __restrict__ T16,
                                                       const int4* __restrict__ tile_info,
                                                       const int64_t* __restrict__ off, const int64_t* __restrict__ ld,
                                                       const int32_t* __restrict__ blk_N, int64_t n_tiles,
                                                       __half* __restrict__ A) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_tiles * kTcRows * 8) return;
  const int64_t tile = t / (kTcRows * 8);
  const int row = int((t / 8) % kTcRows), g = int(t % 8);
  const int4 info = tile_info[tile];
  const int i = info.x, N = blk_N[i];
  const int r = info.y * kTcRows + row;
  __half h[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int n = info.z * 2 * kTcCols + 8 * g + q;
    h[q] = (r < N && n < N) ? __high2half(T16[off[i] + int64_t(r) * ld[i] + n]) : __float2half_rn(0.f);
  }
  *reinterpret_cast<uint4*>(A + tc_tile_index(tile, 1, 0, row, 8 * g)) = *reinterpret_cast<const uint4*>(h);
}

// Real input chunks of the Type-2 apply: thread = (chunk, column col, group g
// of 8 entries); column 4 c + 2 t + f holds part f (0: re, 1: im) of u_t of
// right-hand side c0 + c, as FP16 hi / lo after the column's scaling
__global__ void __launch_bounds__(256) k_tc_build_b_real(const float* __restrict__ x, int64_t ldx, int c0, int nc,
                                                         int nb, const int2* __restrict__ chunk_info, int64_t n_chunks,
                                                         const int32_t* __restrict__ blk_N,
                                                         const int64_t* __restrict__ blk_dof_off,
                                                         const unsigned* __restrict__ colmax, __half* __restrict__ B) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_chunks * nb * 8) return;
  const int64_t chunk = t / (int64_t(nb) * 8);
  const int col = int((t / 8) % nb), g = int(t % 8);
  const int c = col >> 2, slot = (col >> 1) & 1, part = col & 1;
  __half hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) hi[q] = lo[q] = __float2half_rn(0.f);
  if (c < nc) {
    const int2 info = chunk_info[chunk];
    const int N = blk_N[info.x];
    const float s = tc_scale(colmax[c]);
    const float* xc = x + 2 * (int64_t(c0 + c) * ldx + blk_dof_off[info.x] + int64_t(slot) * N) + part;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int n = info.y * 2 * kTcCols + 8 * g + q;
      const float v = n < N ? xc[2 * int64_t(n)] : 0.f;
      tc_split(v * s, hi[q], lo[q]);
    }
  }
  *reinterpret_cast<uint4*>(B + tc_b_index(chunk, 0, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(B + tc_b_index(chunk, 1, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(lo);
}

// lanes per row of the combines: the pass's right-hand sides rounded up to a
// power of two (at least 4), so that one warp takes 32 / lanes rows
__host__ __device__ constexpr int tc_row_lanes(int nc) { return nc <= 4 ? 4 : nc <= 8 ? 8 : nc <= 16 ? 16 : 32; }

// z rows of the block-OSRC apply (one warp per global row, lane = right-hand
// side): the row's pieces of T~ r_D and T~ r_N summed in order and unscaled,
// then z_D = rho^-1 T~ r_N, z_N = -rho T~ r_D with the per-block coefficients
// of the FP16 copy (s_i rho, s_i / rho).  IM (Type 2): the pieces hold
// R r_D and R r_N, and T~ r = i R r.
template <int NB, bool IM = false>
__global__ void __launch_bounds__(256) k_os_tc_combine(
    const float* __restrict__ part, const int32_t* __restrict__ row_blk, const int32_t* __restrict__ blk_N,
    const int64_t* __restrict__ blk_dof_off, const int64_t* __restrict__ blk_row_off, const int* __restrict__ blk_unit_base,
    const int* __restrict__ blk_pieces, const unsigned* __restrict__ colmax, const float* __restrict__ cf,
    float* __restrict__ z, int64_t ldz, int c0, int nc, int64_t n_rows) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int L = tc_row_lanes(nc);
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  const int lane = int(gt % L);
  if (row >= n_rows || lane >= nc) return;
  const int i = row_blk[row];
  const int N = blk_N[i];
  const int64_t m = row - blk_row_off[i];
  const int P = blk_pieces[i];
  const int64_t u0 = blk_unit_base[i] + (m >> 7) * P;
  const int lr = int(m & 127);
  float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int p = 0; p < P; ++p) {
    const float4 a = *reinterpret_cast<const float4*>(part + (size_t(u0 + p) * kTcRows + lr) * NB + 4 * lane);
    t.x += a.x;
    t.y += a.y;
    t.z += a.z;
    t.w += a.w;
  }
  const float sc = tcs_inv_scale(colmax[lane]);
  float a0 = t.x * sc, a1 = t.y * sc, a2 = t.z * sc, a3 = t.w * sc;  // T~ r_D, T~ r_N
  if constexpr (IM) {
    const float d0 = a0, d2 = a2;
    a0 = -a1;
    a1 = d0;
    a2 = -a3;
    a3 = d2;
  }
  const float rr = cf[4 * i], ri = cf[4 * i + 1], ir = cf[4 * i + 2], ii = cf[4 * i + 3];
  float* zc = z + 2 * (int64_t(c0 + lane) * ldz + blk_dof_off[i]);
  zc[2 * m] = ir * a2 - ii * a3;
  zc[2 * m + 1] = ir * a3 + ii * a2;
  zc[2 * (N + m)] = -(rr * a0 - ri * a1);
  zc[2 * (N + m) + 1] = -(rr * a1 + ri * a0);
}

// colmax[c] = max |re|, |im| of input column c0 + c (n complex entries)
__global__ void k_tc_colmax(const float* __restrict__ x, int64_t ldx, int64_t n, int c0, unsigned* __restrict__ colmax) {
  const int c = blockIdx.y;
  const float2* xc = reinterpret_cast<const float2*>(x + 2 * int64_t(c0 + c) * ldx);
  float m = 0.f;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const float2 v = xc[k];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(colmax + c, __float_as_uint(m));
}

// Input chunks: thread = (chunk, column col, group g of 4 complex entries);
// column 4 c + 2 t + f holds form f of u_t of right-hand side c0 + c.
__global__ void __launch_bounds__(256) k_tc_build_b(const float* __restrict__ x, int64_t ldx, int c0, int nc, int nb,
                                                    const int2* __restrict__ chunk_info, int64_t n_chunks,
                                                    const int32_t* __restrict__ blk_N,
                                                    const int64_t* __restrict__ blk_dof_off,
                                                    const unsigned* __restrict__ colmax, __half* __restrict__ B) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_chunks * nb * 8) return;
  const int64_t chunk = t / (int64_t(nb) * 8);
  const int col = int((t / 8) % nb), g = int(t % 8);
  const int c = col >> 2, slot = (col >> 1) & 1, form = col & 1;
  __half hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) hi[q] = lo[q] = __float2half_rn(0.f);
  if (c < nc) {
    const int2 info = chunk_info[chunk];
    const int N = blk_N[info.x];
    const float s = tc_scale(colmax[c]);
    const float2* xc = reinterpret_cast<const float2*>(x + 2 * (int64_t(c0 + c) * ldx + blk_dof_off[info.x] +
                                                                 int64_t(slot) * N));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = info.y * kTcCols + 4 * g + q;
      float2 v = make_float2(0.f, 0.f);
      if (n < N) v = xc[n];
      const float a = form == 0 ? v.x : v.y, b = form == 0 ? -v.y : v.x;
      tc_split(a * s, hi[2 * q], lo[2 * q]);
      tc_split(b * s, hi[2 * q + 1], lo[2 * q + 1]);
    }
  }
  *reinterpret_cast<uint4*>(B + tc_b_index(chunk, 0, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(hi);
  *reinterpret_cast<uint4*>(B + tc_b_index(chunk, 1, col, 8 * g, nb)) = *reinterpret_cast<const uint4*>(lo);
}

template <int NB>
struct TcCfg {
  static constexpr int SA = kTcParts * kTcRows * 128;      // operator tile bytes (64 KB)
  static constexpr int SBB = 2 * NB * 128;                  // input chunk bytes (hi + lo)
  static constexpr int SB = SA + SBB;                       // stage bytes (a multiple of 1024)
  static constexpr int S0 = (220 * 1024) / SB;
  static constexpr int S = S0 > 4 ? 4 : S0;
  static constexpr uint32_t TMEM = 4 * NB < 32 ? 32 : 4 * NB;  // two buffers of 2 NB columns
  static constexpr size_t smem = size_t(S) * SB + 1024 + 256;
  static_assert(S >= 2, "the stage ring needs two stages");
  static_assert(smem <= 232448, "shared memory above the per-CTA limit");
  static_assert(SB % 1024 == 0, "stages must keep the 1024-byte alignment of the swizzled tiles");
};

constexpr uint64_t kTcWaitNs = 500000000ull;

template <int NB>
__global__ void __launch_bounds__(192, 1) k_mv_tc(const __grid_constant__ CUtensorMap amap,
                                                  const __grid_constant__ CUtensorMap bmap,
                                                  const int4* __restrict__ units, const int* __restrict__ sched,
                                                  const int* __restrict__ sched_off,
                                                  const int64_t* __restrict__ blk_tile_base,
                                                  const int* __restrict__ blk_nkc,
                                                  const int64_t* __restrict__ blk_chunk_base, float* __restrict__ part,
                                                  unsigned* __restrict__ err) {
  using C = TcCfg<NB>;
  constexpr int S = C::S, SB = C::SB, SA = C::SA;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(S) * SB);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q_begin = sched_off[blockIdx.x], q_end = sched_off[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tslot, C::TMEM);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch_map(&amap);
      tma_prefetch_map(&bmap);
      const uint64_t pol_a = l2_policy_evict_first(), pol_b = l2_policy_evict_last();
      int k = 0;
      bool ok = true;
      for (int q = q_begin; q < q_end && ok; ++q) {
        const int4 U = units[sched[q]];
        const int64_t tb = blk_tile_base[U.x] + int64_t(U.y) * blk_nkc[U.x];
        const int64_t cb = blk_chunk_base[U.x];
        for (int kc = U.z; kc < U.w; ++kc, ++k) {
          const int st = k % S;
          if (!mbar_wait_bounded(&empty[st], (uint32_t(k / S) & 1u) ^ 1u, kTcWaitNs)) {
            atomicExch(err, 1u);
            ok = false;
            break;
          }
          unsigned char* sa = smem + size_t(st) * SB;
          mbar_arrive_expect_tx(&full[st], uint32_t(SB));
          tma_load_4d(sa, &amap, 0, 0, 0, int(tb + kc), &full[st], pol_a);
          tma_load_4d(sa + SA, &bmap, 0, 0, 0, int(cb + kc), &full[st], pol_b);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16_m128(NB);
      int k = 0, ub = 0;
      bool ok = true;
      for (int q = q_begin; q < q_end && ok; ++q, ++ub) {
        const int4 U = units[sched[q]];
        const int buf = ub & 1;
        if (!mbar_wait_bounded(&tempty[buf], (uint32_t(ub >> 1) & 1u) ^ 1u, kTcWaitNs)) {
          atomicExch(err, 1u);
          break;
        }
        tc_fence_after();
        const uint32_t dT = tmem + uint32_t(buf * 2 * NB), dK = dT + uint32_t(NB);
        for (int kc = U.z; kc < U.w; ++kc, ++k) {
          const int st = k % S;
          if (!mbar_wait_bounded(&full[st], uint32_t(k / S) & 1u, kTcWaitNs)) {
            atomicExch(err, 1u);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + size_t(st) * SB), sb = sa + SA;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t th = sw128_desc(sa + kk * 32), tl = sw128_desc(sa + 16384 + kk * 32);
            const uint64_t kh = sw128_desc(sa + 32768 + kk * 32), kl = sw128_desc(sa + 49152 + kk * 32);
            const uint64_t bh = sw128_desc(sb + kk * 32), bl = sw128_desc(sb + NB * 128 + kk * 32);
            const uint32_t acc = (kc != U.z || kk != 0) ? 1u : 0u;
            tc_mma_f16(dT, th, bh, idesc, acc);
            tc_mma_f16(dT, th, bl, idesc, 1u);
            tc_mma_f16(dT, tl, bh, idesc, 1u);
            tc_mma_f16(dK, kh, bh, idesc, acc);
            tc_mma_f16(dK, kh, bl, idesc, 1u);
            tc_mma_f16(dK, kl, bh, idesc, 1u);
          }
          tc_commit(&empty[st]);  // the stage is free once these MMAs have read it
        }
        if (ok) tc_commit(&tfull[buf]);
      }
    }
  } else {
    // epilogue: warps 2..5 cover the four TMEM lane quarters
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
    int ub = 0;
    for (int q = q_begin; q < q_end; ++q, ++ub) {
      const int buf = ub & 1;
      if (!mbar_wait_bounded(&tfull[buf], uint32_t(ub >> 1) & 1u, kTcWaitNs)) {
        if (lane == 0) atomicExch(err, 1u);
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + (uint32_t(32 * quarter) << 16) + uint32_t(buf * 2 * NB);
      float* dst = part + (size_t(sched[q]) * kTcRows + row) * (2 * NB);
#pragma unroll
      for (int c0 = 0; c0 < 2 * NB; c0 += 16) {
        float v[16];
        tmem_ld16(ta + uint32_t(c0), v);
        float4* d4 = reinterpret_cast<float4*>(dst + c0);
        d4[0] = make_float4(v[0], v[1], v[2], v[3]);
        d4[1] = make_float4(v[4], v[5], v[6], v[7]);
        d4[2] = make_float4(v[8], v[9], v[10], v[11]);
        d4[3] = make_float4(v[12], v[13], v[14], v[15]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM);
  }
}

// y rows (one warp per global row, lane = right-hand side c < nc): the row's
// unit pieces summed in order, unscaled, then the epilogue of Eq. 16 with
// the exchange rows (FP32), as in the FMA stream's combine
template <int NB>
__global__ void __launch_bounds__(256) k_mv_tc_combine(
    const float* __restrict__ part, const int32_t* __restrict__ row_blk, const int32_t* __restrict__ blk_N,
    const int64_t* __restrict__ blk_dof_off, const int64_t* __restrict__ blk_row_off, const int* __restrict__ blk_unit_base,
    const int* __restrict__ blk_pieces, const unsigned* __restrict__ amax, const unsigned* __restrict__ colmax,
    const XEntry* __restrict__ xe, const float* __restrict__ xval32, const float* __restrict__ rho32,
    const float* __restrict__ x, int64_t ldx, float* __restrict__ y, int64_t ldy, int c0, int nc, int64_t n_rows) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  const int L = tc_row_lanes(nc);
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t row = gt / L;
  const int lane = int(gt % L);
  if (row >= n_rows || lane >= nc) return;
  const int i = row_blk[row];
  const int N = blk_N[i];
  const int64_t m = row - blk_row_off[i];
  const int P = blk_pieces[i];
  const int64_t u0 = blk_unit_base[i] + (m >> 7) * P;
  const int lr = int(m & 127);
  float4 t = make_float4(0.f, 0.f, 0.f, 0.f), k = t;
  for (int p = 0; p < P; ++p) {
    const float* pr = part + (size_t(u0 + p) * kTcRows + lr) * (2 * NB);
    const float4 a = *reinterpret_cast<const float4*>(pr + 4 * lane);
    const float4 b = *reinterpret_cast<const float4*>(pr + NB + 4 * lane);
    t.x += a.x;
    t.y += a.y;
    t.z += a.z;
    t.w += a.w;
    k.x += b.x;
    k.y += b.y;
    k.z += b.z;
    k.w += b.w;
  }
  const float sc = tc_inv_scale(amax[i]) * tc_inv_scale(colmax[lane]);
  // T u_D, T u_N, K u_D, K u_N
  const float tDr = t.x * sc, tDi = t.y * sc, tNr = t.z * sc, tNi = t.w * sc;
  const float kDr = k.x * sc, kDi = k.y * sc, kNr = k.z * sc, kNi = k.w * sc;
  const float rr = rho32[4 * i], ri = rho32[4 * i + 1], ir = rho32[4 * i + 2], ii = rho32[4 * i + 3];
  const int col = c0 + lane;
  const float* xc = x + 2 * int64_t(col) * ldx;
  float yDr = 2.f * (kDr + (tNr * ir - tNi * ii));
  float yDi = 2.f * (kDi + (tNr * ii + tNi * ir));
  float yNr = 2.f * (kNr - (tDr * rr - tDi * ri));
  float yNi = 2.f * (kNi - (tDr * ri + tDi * rr));
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const XEntry X = xe[6 * row + e];
    const float xv = xval32[6 * row + e];
    const int Nj = X.ab >> 4;
    yDr += xv * xc[2 * int64_t(X.col)];
    yDi += xv * xc[2 * int64_t(X.col) + 1];
    yNr += xv * xc[2 * (int64_t(X.col) + Nj)];
    yNi += xv * xc[2 * (int64_t(X.col) + Nj) + 1];
  }
  float* yc = y + 2 * (int64_t(col) * ldy + blk_dof_off[i]);
  yc[2 * m] = yDr;
  yc[2 * m + 1] = yDi;
  yc[2 * (N + m)] = yNr;
  yc[2 * (N + m) + 1] = yNi;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q{};
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  MTF_REQUIRE(fn != nullptr, MTF_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// 4-D FP16 map {64, rows, parts, count} over contiguous boxes of
// rows x parts x 128 bytes, loaded with the 128-byte swizzle: whole boxes, or
// (box_parts = 1) only the first part of each box
static void encode_map(void* map, const void* base, int rows, int parts, int box_parts, int64_t count) {
  CUtensorMap* m = static_cast<CUtensorMap*>(map);
  MTF_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0 && count > 0 && count < (int64_t(1) << 31), MTF_ERR_ARG,
              "tensor map base must be 16-byte aligned");
  const cuuint64_t dims[4] = {64, cuuint64_t(rows), cuuint64_t(parts), cuuint64_t(count)};
  const cuuint64_t strides[3] = {128, cuuint64_t(rows) * 128, cuuint64_t(rows) * parts * 128};
  const cuuint32_t box[4] = {64, cuuint32_t(rows), cuuint32_t(box_parts), 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = tensor_map_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void*>(base), dims, strides,
                                          box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  MTF_REQUIRE(r == CUDA_SUCCESS, MTF_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(int(r)));
}
void tc_encode_map(void* map, const void* base, int rows, int parts, int64_t count) {
  encode_map(map, base, rows, parts, parts, count);
}
void tc_encode_map_first(void* map, const void* base, int rows, int parts, int64_t count) {
  encode_map(map, base, rows, parts, 1, count);
}

template <class T>
static void upload_vec(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
  d.alloc(std::max<size_t>(h.size(), 1));
  if (!h.empty()) MTF_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

static void tc_plan_tables(mtf_system sys, TcMatvec& t, cudaStream_t s) {
  if (t.planned) return;
  mtf_mesh m = sys->mesh;
  int dev = 0, sms = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  MTF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  t.n_cta = std::max(1, t.grid > 0 ? std::min(t.grid, sms) : sms);
  std::vector<int> Ns(m->nd);
  for (int i = 0; i < m->nd; ++i) Ns[i] = m->blk[i].N;
  const std::string why = plan_tc(Ns, t.n_cta, t.plan, t.waves, t.min_len);
  MTF_REQUIRE(why.empty(), MTF_ERR_MESH, why);
  const TcPlan& p = t.plan;
  std::vector<int4> units(p.units.size()), tinfo(size_t(p.n_tiles));
  std::vector<int2> cinfo(size_t(p.n_chunks));
  std::vector<int> ubase(m->nd), pieces(m->nd), nkc(m->nd);
  std::vector<int64_t> tbase(m->nd), cbase(m->nd);
  for (size_t u = 0; u < p.units.size(); ++u)
    units[u] = make_int4(p.units[u].blk, p.units[u].mt, p.units[u].kc0, p.units[u].kc1);
  for (int i = 0; i < m->nd; ++i) {
    const TcBlock& b = p.blocks[size_t(i)];
    ubase[i] = b.unit_base;
    pieces[i] = b.pieces;
    nkc[i] = b.n_kc;
    tbase[i] = b.tile_base;
    cbase[i] = b.chunk_base;
    for (int mt = 0; mt < b.n_mt; ++mt)
      for (int kc = 0; kc < b.n_kc; ++kc) tinfo[size_t(b.tile_base + int64_t(mt) * b.n_kc + kc)] = make_int4(i, mt, kc, 0);
    for (int kc = 0; kc < b.n_kc; ++kc) cinfo[size_t(b.chunk_base + kc)] = make_int2(i, kc);
  }
  upload_vec(t.units, units, s);
  std::vector<int4> uab(p.units.size());
  for (size_t u = 0; u < p.units.size(); ++u) {
    const TcBlock& b = p.blocks[size_t(p.units[u].blk)];
    uab[u] = make_int4(int(b.tile_base + int64_t(p.units[u].mt) * b.n_kc), int(b.chunk_base), p.units[u].kc0,
                       p.units[u].kc1);
  }
  MTF_REQUIRE(p.n_tiles < (int64_t(1) << 31), MTF_ERR_MESH, "mesh too large for the tensor-core tables");
  upload_vec(t.units_ab, uab, s);
  upload_vec(t.tile_info, tinfo, s);
  upload_vec(t.chunk_info, cinfo, s);
  upload_vec(t.sched, p.sched, s);
  upload_vec(t.sched_off, p.sched_off, s);
  upload_vec(t.blk_unit_base, ubase, s);
  upload_vec(t.blk_pieces, pieces, s);
  upload_vec(t.blk_nkc, nkc, s);
  upload_vec(t.blk_tile_base, tbase, s);
  upload_vec(t.blk_chunk_base, cbase, s);
  t.amax.alloc(size_t(m->nd));
  t.colmax.alloc(32);
  MTF_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
  t.planned = true;
}

// units, tiles and chunks of the Type-2 block-OSRC apply: the matvec's
// launch plan (CTAs, waves, piece length) over chunks of 64 real columns.
// With the defaults a real row tile has half the chunks of a complex one, so
// the plan asks for 2 units per CTA instead of 4: whole row tiles on large
// systems, which keeps the per-unit epilogue and partial sums from
// dominating the halved stream.
static void tc_osr_plan_tables(mtf_system sys, TcMatvec& t, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  TcMatvec::Real& o = t.osr;
  std::vector<int> Ns(m->nd);
  for (int i = 0; i < m->nd; ++i) Ns[i] = m->blk[i].N;
  const std::string why = plan_tc(Ns, t.n_cta, o.plan, t.waves > 0 ? t.waves : 2, t.min_len, 2 * kTcCols);
  MTF_REQUIRE(why.empty(), MTF_ERR_MESH, why);
  const TcPlan& p = o.plan;
  MTF_REQUIRE(p.n_tiles < (int64_t(1) << 31), MTF_ERR_MESH, "mesh too large for the tensor-core tables");
  std::vector<int4> uab(p.units.size()), tinfo(size_t(p.n_tiles));
  std::vector<int2> cinfo(size_t(p.n_chunks));
  std::vector<int> ubase(m->nd), pieces(m->nd);
  for (size_t u = 0; u < p.units.size(); ++u) {
    const TcBlock& b = p.blocks[size_t(p.units[u].blk)];
    uab[u] = make_int4(int(b.tile_base + int64_t(p.units[u].mt) * b.n_kc), int(b.chunk_base), p.units[u].kc0,
                       p.units[u].kc1);
  }
  for (int i = 0; i < m->nd; ++i) {
    const TcBlock& b = p.blocks[size_t(i)];
    ubase[i] = b.unit_base;
    pieces[i] = b.pieces;
    for (int mt = 0; mt < b.n_mt; ++mt)
      for (int kc = 0; kc < b.n_kc; ++kc) tinfo[size_t(b.tile_base + int64_t(mt) * b.n_kc + kc)] = make_int4(i, mt, kc, 0);
    for (int kc = 0; kc < b.n_kc; ++kc) cinfo[size_t(b.chunk_base + kc)] = make_int2(i, kc);
  }
  upload_vec(o.units_ab, uab, s);
  upload_vec(o.tile_info, tinfo, s);
  upload_vec(o.chunk_info, cinfo, s);
  upload_vec(o.sched, p.sched, s);
  upload_vec(o.sched_off, p.sched_off, s);
  upload_vec(o.blk_unit_base, ubase, s);
  upload_vec(o.blk_pieces, pieces, s);
  MTF_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
  o.planned = true;
}

bool tc_matvec_enabled(mtf_system sys) {
  return sys->opt.precision == MTF_PREC_MIXED && sys->opt.mv_tensor && sys->tc && sys->tc->built;
}

bool tc_wide_apply(mtf_system sys, int nrhs) {
  return nrhs > kFmaPassRhs && tc_matvec_enabled(sys) && !sys->tc->prefer_fma;
}

void tc_set_plan(mtf_system sys, int waves, int min_len, int grid, bool prefer_fma, cudaStream_t s) {
  MTF_REQUIRE(tc_matvec_enabled(sys), MTF_ERR_ARG, "tensor-core matvec not built for this system");
  TcMatvec& t = *sys->tc;
  t.prefer_fma = prefer_fma;
  if (t.waves == waves && t.min_len == min_len && t.grid == grid && t.planned) return;
  MTF_CUDA(cudaStreamSynchronize(s));  // launches queued with the old tables have finished
  t.waves = waves;
  t.min_len = min_len;
  t.grid = grid;
  t.planned = false;
  tc_plan_tables(sys, t, s);
  if (t.osr.planned) tc_osr_plan_tables(sys, t, s);  // same tile order, new units
}

// FP16 hi / lo tiled copy of the FP32-stored {T, K}, rebuilt after every
// mixed-precision assembly
void tc_build_operator(mtf_system sys, cudaStream_t s) {
  if (!sys->opt.mv_tensor) return;
  if (!sys->tc) sys->tc = new TcMatvec();
  TcMatvec& t = *sys->tc;
  mtf_mesh m = sys->mesh;
  tc_plan_tables(sys, t, s);
  const size_t nh = size_t(t.plan.n_tiles) * size_t(kTcTileHalves);
  if (t.A.n != nh) {
    t.A.alloc(nh);
    t.amap_ptr = nullptr;
  }
  MTF_CUDA(cudaMemsetAsync(t.amax.p, 0, size_t(m->nd) * sizeof(unsigned), s));
  MTF_LAUNCH(KID_TC_TILE, s, k_tc_blkmax<<<dim3(256, unsigned(m->nd)), 256, 0, s>>>(
      reinterpret_cast<const float4*>(sys->d_TK32.p), m->d_blk_mat_off.p, m->d_blk_N.p, t.amax.p));
  const int64_t nthr = t.plan.n_tiles * kTcRows * 8;
  MTF_LAUNCH(KID_TC_TILE, s, k_tc_tile_a<<<unsigned((nthr + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const float4*>(sys->d_TK32.p), t.tile_info.p, m->d_blk_mat_off.p, m->d_blk_N.p, t.amax.p,
      t.plan.n_tiles, t.A.p));
  if (t.amap_ptr != t.A.p) {
    tc_encode_map(&t.amap, t.A.p, kTcRows, kTcParts, t.plan.n_tiles);
    t.amap_ptr = t.A.p;
  }
  t.built = true;
}

// input chunks (hi, lo) of columns c0 .. c0 + nc - 1 of x in t.B, their
// scales in t.colmax, and the B tensor map for width NB
template <int NB>
static void tc_build_inputs(mtf_system sys, TcMatvec& t, const float* x, int64_t ldx, int c0, int nc, int kid,
                            cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const TcPlan& p = t.plan;
  const size_t bh = size_t(p.n_chunks) * 2 * NB * 64;
  if (t.B.n < bh) {
    t.B.alloc(size_t(p.n_chunks) * 2 * 128 * 64);  // room for the widest pass
    t.bmap_ptr = nullptr;
  }
  if (t.bmap_ptr != t.B.p || t.bmap_nb != NB) {
    tc_encode_map(&t.bmap, t.B.p, NB, 2, p.n_chunks);
    t.bmap_ptr = t.B.p;
    t.bmap_nb = NB;
  }
  const size_t np = p.units.size() * kTcRows * 2 * NB;
  if (t.part.n < np) t.part.alloc(size_t(p.units.size()) * kTcRows * 2 * 128);
  MTF_CUDA(cudaMemsetAsync(t.colmax.p, 0, 32 * sizeof(unsigned), s));
  MTF_LAUNCH(kid, s, k_tc_colmax<<<dim3(64, unsigned(nc)), 256, 0, s>>>(x, ldx, m->n_total, c0, t.colmax.p));
  const int64_t nthr = p.n_chunks * NB * 8;
  MTF_LAUNCH(kid, s, launch_pdl(k_tc_build_b, dim3(unsigned((nthr + 255) / 256)), dim3(256), 0, s,
      x, ldx, c0, nc, NB, t.chunk_info.p, p.n_chunks, m->d_blk_N.p, m->d_blk_dof_off.p, t.colmax.p, t.B.p));
}

template <int NB>
static void mv_tc_pass(mtf_system sys, TcMatvec& t, const float* x, int64_t ldx, float* y, int64_t ldy, int c0, int nc,
                       cudaStream_t s) {
  using Cfg = TcCfg<NB>;
  mtf_mesh m = sys->mesh;
  tc_build_inputs<NB>(sys, t, x, ldx, c0, nc, KID_MVTC_PREP, s);
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_mv_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem)));
    opted.fetch_or(bit);
  }
  stream_prepare(sys, s);
  // every stored {T, K} entry once (16 bytes: FP16 hi + lo of four reals)
  // and the pass's FP16 hi + lo input chunks once
  prof_bytes(KID_MVTC, double(m->n_mat) * 16.0 + double(m->n_total) * nc * 8.0);
  MTF_LAUNCH(KID_MVTC, s, k_mv_tc<NB><<<unsigned(t.n_cta), 192, Cfg::smem, s>>>(
      t.amap, t.bmap, t.units.p, t.sched.p, t.sched_off.p, t.blk_tile_base.p, t.blk_nkc.p, t.blk_chunk_base.p,
      t.part.p, sys->d_mv_ctl.p + 2));
  const unsigned gc = unsigned((m->n_rows * tc_row_lanes(nc) + 255) / 256);
  MTF_LAUNCH(KID_MVTC_COMBINE, s, launch_pdl(k_mv_tc_combine<NB>, dim3(gc), dim3(256), 0, s,
      t.part.p, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p, m->d_blk_row_off.p, t.blk_unit_base.p,
      t.blk_pieces.p, t.amax.p, t.colmax.p, m->d_xent.p, sys->d_xval32.p, sys->d_rho32.p, x, ldx, y, ldy, c0, nc,
      m->n_rows));
}

// FP16 T~ tiles of the block-OSRC apply, rebuilt from the FP16 copy of T~
// (osrc.cu) after every assembly
void tc_build_osrc(mtf_system sys, const std::vector<int64_t>& ld16, cudaStream_t s) {
  if (!sys->opt.mv_tensor || sys->opt.precision != MTF_PREC_MIXED || !sys->d_osrc_T16.p) return;
  if (!sys->tc) sys->tc = new TcMatvec();
  TcMatvec& t = *sys->tc;
  mtf_mesh m = sys->mesh;
  tc_plan_tables(sys, t, s);
  upload_vec(t.os_off, m->os16_off_h, s);
  upload_vec(t.os_ld, ld16, s);
  if (sys->opt.osrc_type == 2) {
    // Type 2: tiles of R = Im T~ (64 real columns per tile row)
    TcMatvec::Real& o = t.osr;
    if (!o.planned) tc_osr_plan_tables(sys, t, s);
    const size_t nr = size_t(o.plan.n_tiles) * kTcRows * 64;
    if (o.A.n != nr) {
      o.A.alloc(nr);
      o.amap_ptr = nullptr;
    }
    const int64_t nthr = o.plan.n_tiles * kTcRows * 8;
    MTF_LAUNCH(KID_TC_TILE, s, k_tc_tile_os_im<<<unsigned((nthr + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const __half2*>(sys->d_osrc_T16.p), o.tile_info.p, t.os_off.p, t.os_ld.p, m->d_blk_N.p,
        o.plan.n_tiles, o.A.p));
    if (o.amap_ptr != o.A.p) {
      tc_encode_map(&o.amap, o.A.p, kTcRows, 1, o.plan.n_tiles);
      o.amap_ptr = o.A.p;
    }
    MTF_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
    t.os_built = true;
    return;
  }
  const size_t nh = size_t(t.plan.n_tiles) * kTcRows * 64;
  if (t.Aos.n != nh) {
    t.Aos.alloc(nh);
    t.osmap_ptr = nullptr;
  }
  const int64_t nthr = t.plan.n_tiles * kTcRows * 8;
  MTF_LAUNCH(KID_TC_TILE, s, k_tc_tile_os<<<unsigned((nthr + 255) / 256), 256, 0, s>>>(
      reinterpret_cast<const __half2*>(sys->d_osrc_T16.p), t.tile_info.p, t.os_off.p, t.os_ld.p, m->d_blk_N.p,
      t.plan.n_tiles, t.Aos.p));
  if (t.osmap_ptr != t.Aos.p) {
    tc_encode_map(&t.osmap, t.Aos.p, kTcRows, 1, t.plan.n_tiles);
    t.osmap_ptr = t.Aos.p;
  }
  MTF_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
  t.os_built = true;
}

bool tc_osrc_enabled(mtf_system sys) {
  return sys->opt.precision == MTF_PREC_MIXED && sys->opt.mv_tensor && sys->opt.osrc_half && sys->tc &&
         sys->tc->os_built;
}

template <int NB>
static void os_tc_pass(mtf_system sys, TcMatvec& t, const float* r, int64_t ldr, float* z, int64_t ldz, int c0, int nc,
                       cudaStream_t s) {
  using Cfg = TcsCfg<1, NB>;
  mtf_mesh m = sys->mesh;
  tc_build_inputs<NB>(sys, t, r, ldr, c0, nc, KID_OSRC, s);
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_tc_stream<1, NB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem)));
    opted.fetch_or(bit);
  }
  stream_prepare(sys, s);
  // every stored FP16 T~ entry once and the pass's inputs once
  prof_bytes(KID_OSRC, double(m->n_mat) * 4.0 + double(m->n_total) * nc * 8.0);
  TcUnits units;
  units.list = t.units_ab.p;
  MTF_LAUNCH(KID_OSRC, s, k_tc_stream<1, NB, 0><<<unsigned(t.n_cta), 192, Cfg::smem, s>>>(
      t.osmap, t.bmap, units, int(t.plan.units.size()), t.sched.p, t.sched_off.p, t.part.p, nullptr, 0, 0, 0, nullptr,
      sys->d_mv_ctl.p + 2, TcTtOut{}));
  const unsigned gc = unsigned((m->n_rows * tc_row_lanes(nc) + 255) / 256);
  MTF_LAUNCH(KID_OSCOMBINE, s, launch_pdl(k_os_tc_combine<NB>, dim3(gc), dim3(256), 0, s,
      t.part.p, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p, m->d_blk_row_off.p, t.blk_unit_base.p,
      t.blk_pieces.p, t.colmax.p, sys->d_os_coef16.p, z, ldz, c0, nc, m->n_rows));
}

// The Type-2 pass: real input chunks of the pass's columns, one stream over
// the FP16 tiles of R (2 bytes per stored entry), and the combine with
// T~ r = i R r
template <int NB>
static void os_tc_pass_real(mtf_system sys, TcMatvec& t, const float* r, int64_t ldr, float* z, int64_t ldz, int c0,
                            int nc, cudaStream_t s) {
  using Cfg = TcsCfg<1, NB>;
  mtf_mesh m = sys->mesh;
  TcMatvec::Real& o = t.osr;
  const TcPlan& p = o.plan;
  if (o.B.n < size_t(p.n_chunks) * 2 * NB * 64) {
    o.B.alloc(size_t(p.n_chunks) * 2 * 128 * 64);  // room for the widest pass
    o.bmap_ptr = nullptr;
  }
  if (o.bmap_ptr != o.B.p || o.bmap_nb != NB) {
    tc_encode_map(&o.bmap, o.B.p, NB, 2, p.n_chunks);
    o.bmap_ptr = o.B.p;
    o.bmap_nb = NB;
  }
  if (o.part.n < p.units.size() * kTcRows * NB) o.part.alloc(p.units.size() * kTcRows * 128);
  MTF_CUDA(cudaMemsetAsync(t.colmax.p, 0, 32 * sizeof(unsigned), s));
  MTF_LAUNCH(KID_OSRC, s, k_tc_colmax<<<dim3(64, unsigned(nc)), 256, 0, s>>>(r, ldr, m->n_total, c0, t.colmax.p));
  const int64_t nthr = p.n_chunks * NB * 8;
  MTF_LAUNCH(KID_OSRC, s, launch_pdl(k_tc_build_b_real, dim3(unsigned((nthr + 255) / 256)), dim3(256), 0, s,
      r, ldr, c0, nc, NB, o.chunk_info.p, p.n_chunks, m->d_blk_N.p, m->d_blk_dof_off.p, t.colmax.p, o.B.p));
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_tc_stream<1, NB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem)));
    opted.fetch_or(bit);
  }
  stream_prepare(sys, s);
  // every stored FP16 entry of R once and the pass's inputs once
  prof_bytes(KID_OSRC, double(m->n_mat) * 2.0 + double(m->n_total) * nc * 8.0);
  TcUnits units;
  units.list = o.units_ab.p;
  MTF_LAUNCH(KID_OSRC, s, k_tc_stream<1, NB, 0><<<unsigned(t.n_cta), 192, Cfg::smem, s>>>(
      o.amap, o.bmap, units, int(p.units.size()), o.sched.p, o.sched_off.p, o.part.p, nullptr, 0, 0, 0, nullptr,
      sys->d_mv_ctl.p + 2, TcTtOut{}));
  const unsigned gc = unsigned((m->n_rows * tc_row_lanes(nc) + 255) / 256);
  MTF_LAUNCH(KID_OSCOMBINE, s,
             launch_pdl(k_os_tc_combine<NB, true>, dim3(gc), dim3(256), 0, s,
                 o.part.p, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p, m->d_blk_row_off.p, o.blk_unit_base.p,
                 o.blk_pieces.p, t.colmax.p, sys->d_os_coef16.p, z, ldz, c0, nc, m->n_rows));
}

// z = A~ r (block-OSRC, Eq. 19) with the FP16 T~ on the tensor cores, in
// passes of up to 32 right-hand sides (FP32 in and out)
void launch_osrc_apply_tc(mtf_system sys, const float* r, int64_t ldr, float* z, int64_t ldz, int nrhs,
                          cudaStream_t s) {
  MTF_REQUIRE(tc_osrc_enabled(sys), MTF_ERR_ARG, "tensor-core block-OSRC not built for this system");
  TcMatvec& t = *sys->tc;
  MTF_REQUIRE((reinterpret_cast<uintptr_t>(r) & 15) == 0 && (ldr & 1) == 0, MTF_ERR_ARG,
              "tensor-core block-OSRC input columns must be 16-byte aligned");
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int nc = std::min(32, nrhs - c0);
    const int nb = tc_nb(nc);
    if (sys->opt.osrc_type == 2) {
      if (nb == 16) os_tc_pass_real<16>(sys, t, r, ldr, z, ldz, c0, nc, s);
      else if (nb == 32) os_tc_pass_real<32>(sys, t, r, ldr, z, ldz, c0, nc, s);
      else if (nb == 64) os_tc_pass_real<64>(sys, t, r, ldr, z, ldz, c0, nc, s);
      else os_tc_pass_real<128>(sys, t, r, ldr, z, ldz, c0, nc, s);
      continue;
    }
    if (nb == 16) os_tc_pass<16>(sys, t, r, ldr, z, ldz, c0, nc, s);
    else if (nb == 32) os_tc_pass<32>(sys, t, r, ldr, z, ldz, c0, nc, s);
    else if (nb == 64) os_tc_pass<64>(sys, t, r, ldr, z, ldz, c0, nc, s);
    else os_tc_pass<128>(sys, t, r, ldr, z, ldz, c0, nc, s);
  }
}

// y = M x (FP32 in and out) on the tensor cores, in passes of up to 32
// right-hand sides; x and y need 16-byte aligned columns
void launch_matvec_tc(mtf_system sys, const float* x, int64_t ldx, float* y, int64_t ldy, int nrhs, cudaStream_t s) {
  MTF_REQUIRE(tc_matvec_enabled(sys), MTF_ERR_ARG, "tensor-core matvec not built for this system");
  TcMatvec& t = *sys->tc;
  MTF_REQUIRE((reinterpret_cast<uintptr_t>(x) & 15) == 0 && (ldx & 1) == 0, MTF_ERR_ARG,
              "tensor-core matvec input columns must be 16-byte aligned");
  for (int c0 = 0; c0 < nrhs; c0 += 32) {
    const int nc = std::min(32, nrhs - c0);
    const int nb = tc_nb(nc);
    if (nb == 16) mv_tc_pass<16>(sys, t, x, ldx, y, ldy, c0, nc, s);
    else if (nb == 32) mv_tc_pass<32>(sys, t, x, ldx, y, ldy, c0, nc, s);
    else if (nb == 64) mv_tc_pass<64>(sys, t, x, ldx, y, ldy, c0, nc, s);
    else mv_tc_pass<128>(sys, t, x, ldx, y, ldy, c0, nc, s);
  }
}

}  // namespace mtf
