// Bulk-copy tiled streaming kernel of the FP32 operator applies: the block
// matvec (entries {T, K}: two complex FP32 values, ENT = 2) and the
// block-OSRC apply (entries T~: one complex FP32 value, ENT = 1).
//
// An operator is streamed either from its dense rows (one bulk copy per row
// of a unit) or from a tiled copy in which each unit is one contiguous run
// (toff[u] its byte offset, rows at st_tile_pitch; one bulk copy per unit):
// the bulk-copy count per byte bounds the row-by-row form.
//
// A dense block is cut into work units of st_unit_rows<ENT>() consecutive
// rows x one column piece of at most st_piece_len<ENT>() entries (every row
// of block i in P_i pieces of near-equal length).  One persistent CTA per SM
// takes units blockIdx.x, blockIdx.x + gridDim.x, ...  A producer warp
// fetches, with the TMA engine (cp.async.bulk, one "full" mbarrier per
// stage), the unit's row pieces and the matching slices of the input vectors
// (D and N slots of every right-hand side) into a ring of S shared-memory
// stages; st_consumers<ENT>() consumer warps, st_rpw<ENT>() rows each, read both
// from shared memory, so the input slice is fetched once per unit instead of
// once per row, each value of it read from shared memory serves every row of
// the warp, and no consumer waits on a global load.  Consumers release a
// stage through an "empty" mbarrier.
//
// Per row and right-hand side a consumer forms the partial sums
//   ENT = 2:      T x_D, T x_N, K x_D, K x_N    (8 floats)
//   ENT = 1, 3:   T~ x_D, T~ x_N                (4 floats; T~ in FP32 or FP16)
// reduces them over the warp (recursive halving) and stores them at
// part[(row * pmax + piece) * K + value]; a per-operator combine kernel adds
// each row's pieces in fixed order and applies the epilogue.
//
// Bulk copies need 16-byte aligned addresses and sizes: rows of ENT = 1
// operators are stored with an even row stride and pieces start at even
// columns (the host checks every unit), and input slices are widened to the
// enclosing 16-byte boundaries, which stay inside the vector because vectors
// start at even complex offsets (ld32 even, 16-byte aligned base: checked by
// the host).  Every wait is bounded (~0.5 s): on timeout the kernel sets *err
// and its warps leave.
#pragma once

#include <atomic>

#include <cuda_fp16.h>

#include "bulk.h"
#include "common.h"

namespace mtf {

// tuning (compile-time overridable): bytes of one row piece for 16-byte
// ({T, K}) and 8-byte (T~) entries, shared-memory budget of the stage ring
#ifndef MTF_ST_PIECE_BYTES2
#define MTF_ST_PIECE_BYTES2 4096
#endif
#ifndef MTF_ST_PIECE_BYTES1
#define MTF_ST_PIECE_BYTES1 4096
#endif
#ifndef MTF_ST_PIECE_BYTES3
#define MTF_ST_PIECE_BYTES3 2560
#endif
// consumer warps and rows per consumer warp for the 8- and 4-byte entry
// types (the 16-byte {T, K} entries use 8 warps of two rows).  Measured on
// the split sphere: 8 x 2, 16 x 1 and 8 x 4 run within 4% of each other at
// these piece sizes; smaller pieces are slower (per-unit costs)
#ifndef MTF_ST_CONS1
#define MTF_ST_CONS1 8
#endif
#ifndef MTF_ST_RPW1
#define MTF_ST_RPW1 2
#endif
#ifndef MTF_ST_UNROLL2
#define MTF_ST_UNROLL2 1
#endif
#ifndef MTF_ST_UNROLL1
#define MTF_ST_UNROLL1 8
#endif
#ifndef MTF_ST_UNROLL3
#define MTF_ST_UNROLL3 8
#endif
#ifndef MTF_ST_SMEM_BUDGET
#define MTF_ST_SMEM_BUDGET (220 * 1024)
#endif
constexpr int kStMaxStages = 8;
constexpr int kStSmemBudget = MTF_ST_SMEM_BUDGET;
constexpr uint64_t kStWaitNs = 500000000ull;
// Entry types: ENT = 2: {T, K} as two complex FP32 (16 bytes); ENT = 1: one
// complex FP32 (8 bytes); ENT = 3: one complex FP16 (4 bytes, __half2).
template <int ENT>
__host__ __device__ constexpr int st_eb() {
  return ENT == 2 ? 16 : (ENT == 1 ? 8 : 4);
}
// partial sums per right-hand side and row piece: (T, K) x (x_D, x_N) or
// T x (x_D, x_N), complex
template <int ENT>
__host__ __device__ constexpr int st_nv() {
  return ENT == 2 ? 8 : 4;
}
// entries between consecutive rows of an N x N block: 16-byte aligned rows
template <int ENT>
__host__ __device__ inline int64_t st_row_stride(int N) {
  return ENT == 2 ? N : (ENT == 1 ? N + (N & 1) : (N + 3) & ~3);
}

// consumer warps per CTA, rows per consumer warp and rows per unit
template <int ENT>
__host__ __device__ constexpr int st_consumers() {
  return ENT == 2 ? 8 : MTF_ST_CONS1;
}
template <int ENT>
__host__ __device__ constexpr int st_rpw() {
  return ENT == 2 ? 2 : MTF_ST_RPW1;
}
template <int ENT>
__host__ __device__ constexpr int st_unit_rows() {
  return st_consumers<ENT>() * st_rpw<ENT>();
}
template <int ENT>
__host__ __device__ constexpr int st_threads() {
  return (st_consumers<ENT>() + 1) * 32;
}

// consumer loop unrolling per entry type (measured: the 16-byte entries run
// fastest unrolled once, the 8-byte ones eight times)
template <int ENT>
constexpr int st_unroll() {
  return ENT == 2 ? MTF_ST_UNROLL2 : (ENT == 1 ? MTF_ST_UNROLL1 : MTF_ST_UNROLL3);
}

// entries per piece (one row's slot in a stage)
template <int ENT>
__host__ __device__ constexpr int st_piece_len() {
  return (ENT == 2 ? MTF_ST_PIECE_BYTES2 : (ENT == 1 ? MTF_ST_PIECE_BYTES1 : MTF_ST_PIECE_BYTES3)) / st_eb<ENT>();
}

template <int NC, int ENT>
struct StreamK {
  static constexpr int raw = st_nv<ENT>() * NC;  // partial sums per row piece
  static constexpr int K = raw <= 4 ? 4 : (raw <= 8 ? 8 : (raw <= 16 ? 16 : 32));
  static constexpr int SH = K == 4 ? 3 : (K == 8 ? 2 : (K == 16 ? 1 : 0));  // value index = lane >> SH
  static constexpr int L = st_piece_len<ENT>();
  static constexpr int RB = L * st_eb<ENT>();                                  // bytes of a row slot
  static constexpr int XB = (L + 2) * 8;                                       // bytes of an input-slice slot
  static constexpr int ROWS = st_unit_rows<ENT>();
  static constexpr int SB = ((ROWS * RB + 2 * NC * XB) + 127) / 128 * 128;  // bytes of a stage
  static constexpr int S = (kStSmemBudget / SB) < kStMaxStages ? (kStSmemBudget / SB) : kStMaxStages;
  static constexpr size_t smem = size_t(S) * SB + size_t(S) * (2 * sizeof(uint64_t) + sizeof(int4));
  static_assert(S >= 2, "the stage ring needs at least two stages");
  static_assert(smem <= 232448, "shared memory above the per-CTA limit");
};

// partial sums of one row piece against NC right-hand sides, accumulated into v
template <int NC, int ENT>
__device__ __forceinline__ void st_row_fma(float* v, const unsigned char* rowp, const float2* const* xs, int e) {
  if constexpr (ENT == 2) {
    const float4 a = reinterpret_cast<const float4*>(rowp)[e];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float2 xd = xs[2 * c][e], xn = xs[2 * c + 1][e];
      float* w = v + 8 * c;
      w[0] = fmaf(a.x, xd.x, fmaf(-a.y, xd.y, w[0]));  // T x_D
      w[1] = fmaf(a.x, xd.y, fmaf(a.y, xd.x, w[1]));
      w[2] = fmaf(a.x, xn.x, fmaf(-a.y, xn.y, w[2]));  // T x_N
      w[3] = fmaf(a.x, xn.y, fmaf(a.y, xn.x, w[3]));
      w[4] = fmaf(a.z, xd.x, fmaf(-a.w, xd.y, w[4]));  // K x_D
      w[5] = fmaf(a.z, xd.y, fmaf(a.w, xd.x, w[5]));
      w[6] = fmaf(a.z, xn.x, fmaf(-a.w, xn.y, w[6]));  // K x_N
      w[7] = fmaf(a.z, xn.y, fmaf(a.w, xn.x, w[7]));
    }
  } else {
    float2 a;
    if constexpr (ENT == 1) a = reinterpret_cast<const float2*>(rowp)[e];
    else a = __half22float2(reinterpret_cast<const __half2*>(rowp)[e]);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float2 xd = xs[2 * c][e], xn = xs[2 * c + 1][e];
      float* w = v + 4 * c;
      w[0] = fmaf(a.x, xd.x, fmaf(-a.y, xd.y, w[0]));  // T~ x_D
      w[1] = fmaf(a.x, xd.y, fmaf(a.y, xd.x, w[1]));
      w[2] = fmaf(a.x, xn.x, fmaf(-a.y, xn.y, w[2]));  // T~ x_N
      w[3] = fmaf(a.x, xn.y, fmaf(a.y, xn.x, w[3]));
    }
  }
}

// unit record: {N of the block, global row of the unit's first row, first
// input column (dof offset of the block + first column of the piece),
// len | piece << 12 | rows << 24 (rows <= 64)}; usrc: entry offset of the
// first row's piece
template <int NC, int ENT>
__global__ void __launch_bounds__(st_threads<ENT>(), 1) k_stream_tiles(
    const void* __restrict__ entries, const int4* __restrict__ units, const int64_t* __restrict__ usrc, int n_units,
    int pmax, const float* __restrict__ x32, int64_t ld32, int c0, float* __restrict__ part,
    unsigned* __restrict__ err, const int64_t* __restrict__ toff) {
  using SK = StreamK<NC, ENT>;
  constexpr int RW = st_rpw<ENT>(), ROWS = SK::ROWS;
  constexpr int EB = st_eb<ENT>(), Q = 16 / EB, K = SK::K, SH = SK::SH, RB = SK::RB, XB = SK::XB, SB = SK::SB, S = SK::S;
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(S) * SB);
  uint64_t* empty = full + S;
  int4* meta = reinterpret_cast<int4*>(empty + S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], st_consumers<ENT>());
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == st_consumers<ENT>()) {
    // producer: one lane issues every copy
    if (lane != 0) return;
    const unsigned char* ent = static_cast<const unsigned char*>(entries);
    // the operator is read once per apply: its lines go first out of L2, so
    // the reused vectors and the Krylov basis stay resident
    const uint64_t stream_pol = l2_policy_evict_first();
    // unit records are loaded one unit ahead so that their global round trip
    // overlaps the wait for a free stage
    int4 nrec = make_int4(0, 0, 0, 0);
    int64_t nsrc = 0;
    if (int(blockIdx.x) < n_units) {
      nrec = units[blockIdx.x];
      nsrc = usrc[blockIdx.x];
    }
    int k = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++k) {
      const int4 rec = nrec;
      const int64_t src = nsrc;
      if (u + int(gridDim.x) < n_units) {
        nrec = units[u + gridDim.x];
        nsrc = usrc[u + gridDim.x];
      }
      const int s = k % S;
      if (!mbar_wait_bounded(&empty[s], (uint32_t(k / S) & 1u) ^ 1u, kStWaitNs)) {
        atomicExch(err, 1u);
        return;
      }
      const int N = rec.x, len = rec.w & 0xfff, nrows = (rec.w >> 24) & 0xff;
      const int64_t stride = st_row_stride<ENT>(N);
      const uint32_t rb = uint32_t((len + Q - 1) / Q * Q) * EB;
      // tiled operator: the unit's rows are one contiguous run at the tiled pitch
      const uint32_t pitch = toff ? uint32_t(st_tile_pitch(EB, len)) : uint32_t(RB);
      uint32_t total = toff ? uint32_t(nrows) * pitch : uint32_t(nrows) * rb;
      int64_t xa[2 * NC];
      uint32_t xbytes[2 * NC];
#pragma unroll
      for (int q = 0; q < 2 * NC; ++q) {
        const int64_t a = int64_t(c0 + (q >> 1)) * ld32 + rec.z + (q & 1) * N;
        xa[q] = a & ~int64_t(1);
        xbytes[q] = uint32_t((((a + len + 1) & ~int64_t(1)) - xa[q]) * 8);
        total += xbytes[q];
      }
      meta[s] = rec;
      mbar_arrive_expect_tx(&full[s], total);
      unsigned char* st = smem + size_t(s) * SB;
      if (toff)
        bulk_g2s_hint(st, ent + toff[u], uint32_t(nrows) * pitch, &full[s], stream_pol);
      else
        for (int r = 0; r < nrows; ++r)
          bulk_g2s_hint(st + r * RB, ent + (src + r * stride) * EB, rb, &full[s], stream_pol);
#pragma unroll
      for (int q = 0; q < 2 * NC; ++q)
        bulk_g2s(st + ROWS * RB + q * XB, x32 + 2 * xa[q], xbytes[q], &full[s]);
    }
    return;
  }

  // consumers: warp w owns rows RW w .. RW w + RW - 1 of every unit; each
  // input value read from shared memory feeds all of them
  int k = 0;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++k) {
    const int s = k % S;
    if (!mbar_wait_bounded(&full[s], uint32_t(k / S) & 1u, kStWaitNs)) {
      if (lane == 0) atomicExch(err, 1u);
      return;
    }
    const int4 rec = meta[s];
    const int N = rec.x, len = rec.w & 0xfff, p = (rec.w >> 12) & 0xfff, nrows = (rec.w >> 24) & 0xff;
    const int pitch = toff ? st_tile_pitch(EB, len) : RB;
    const unsigned char* st = smem + size_t(s) * SB;
    const int r0 = RW * warp;
    if (r0 < nrows) {
      const float2* xs[2 * NC];
#pragma unroll
      for (int q = 0; q < 2 * NC; ++q) {
        const int64_t a = int64_t(c0 + (q >> 1)) * ld32 + rec.z + (q & 1) * N;
        xs[q] = reinterpret_cast<const float2*>(st + ROWS * RB + q * XB) + (a & 1);
      }
      float v[RW][K];
      const unsigned char* rowp[RW];
#pragma unroll
      for (int r = 0; r < RW; ++r) {
#pragma unroll
        for (int q = 0; q < K; ++q) v[r][q] = 0.f;
        rowp[r] = st + min(r0 + r, nrows - 1) * pitch;  // repeats of the unit's last row are discarded
      }
#pragma unroll st_unroll<ENT>()
      for (int e = lane; e < len; e += 32) {
#pragma unroll
        for (int r = 0; r < RW; ++r) st_row_fma<NC, ENT>(v[r], rowp[r], xs, e);
      }
#pragma unroll
      for (int r = 0; r < RW; ++r) WarpTransposeSum<K>::run(v[r], lane, 16);
      if ((lane & ((1 << SH) - 1)) == 0) {
#pragma unroll
        for (int r = 0; r < RW; ++r)
          if (r0 + r < nrows) part[(int64_t(rec.y + r0 + r) * pmax + p) * K + (lane >> SH)] = v[r][0];
      }
    }
    // release the stage: order this warp's shared reads before the next bulk write
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// one launch of the tiled streaming kernel for right-hand sides c0 .. c0+NC-1
template <int NC, int ENT>
void launch_stream_tiles(mtf_system sys, const void* entries, const StreamUnits& su, const float* x32, int64_t ld32,
                         int c0, float* part, int kid, cudaStream_t s, bool tiled = false) {
  using SK = StreamK<NC, ENT>;
  MTF_REQUIRE(ld32 % 2 == 0 && (reinterpret_cast<uintptr_t>(x32) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(entries) & 15) == 0,
              MTF_ERR_ARG, "streamed vectors and operators must be 16-byte aligned with an even column stride");
  auto kfn = k_stream_tiles<NC, ENT>;
  // the shared-memory opt-in is set once per device, not on every launch
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load(std::memory_order_relaxed) & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SK::smem)));
    opted.fetch_or(bit);
  }
  MTF_LAUNCH(kid, s,
             launch_pdl(kfn, dim3(unsigned(sys->mv_grid)), dim3(st_threads<ENT>()), SK::smem, s, entries,
                        su.d_units.p, su.d_src.p, int(su.n_units), su.pmax, x32, ld32, c0, part, sys->d_mv_ctl.p + 2,
                        tiled ? su.d_toff.p : static_cast<const int64_t*>(nullptr)));
}

// Sum of the P piece partials of one row (stored contiguously, K per piece)
// for value index lane % K: every lane loads its share independently and the
// lanes holding the same value index are combined in a fixed order.
template <int K>
__device__ __forceinline__ float st_row_total(const float* __restrict__ prow, int P, int lane) {
  float acc = 0.f;
  const int n = P * K;
  for (int j = lane; j < n; j += 32) acc += prow[j];
#pragma unroll
  for (int o = K; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// pieces of a row of N entries (the combine kernels use the same count)
template <int ENT>
__host__ __device__ inline int st_pieces(int N) {
  return N <= 0 ? 1 : (N + st_piece_len<ENT>() - 1) / st_piece_len<ENT>();
}

}  // namespace mtf
