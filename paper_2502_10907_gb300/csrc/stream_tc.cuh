// Tensor-core variant of the streaming block-OSRC apply for the FP16 copy of
// T~ (entry type 3 of stream.cuh).
//
// Per unit (16 consecutive rows x one column piece of a block's T~), the
// complex products T~ x_q for the 2 NC input columns (D and N slot of every
// right-hand side) are one real matrix product: a row of T~ stored as
// interleaved (re, im) halves is a real row of length 2 len, and column q
// becomes two real columns,
//   [x_re, -x_im, ...]  (real part of T~ x_q)   and   [x_im, x_re, ...]  (imaginary part),
// so 16 rows x 8 real columns x 16 real terms is one mma.sync m16n8k16 (FP16
// operands, FP32 accumulation).  The inputs are rounded to FP16 like T~
// itself (2^-11 relative); the preconditioner's output changes by about as
// much as the FP16 copy of T~ changes it, and flexible GMRES takes the
// vectors it applied.
//
// The producer warp works as in stream.cuh (bulk copies into a ring of
// stages, bounded waits), but streams a tiled copy of the FP16 T~ in which
// every unit is one contiguous run: its rows at a pitch of whole k16 chunks
// (8 complex entries, zero past the piece) padded to 16 bytes past a
// 128-byte multiple, so that the eight rows an ldmatrix phase reads fall in
// distinct banks.  One bulk copy per unit instead of one per row: the copy
// count, not DRAM, bounded the row-by-row version (about 90 ns per copy and
// SM, measured).  The 8 consumer
// warps take the piece's k16 chunks in turn, add their 16 x 8 partial tiles
// in shared memory (double-buffered, one named barrier per unit) and store
// the row piece sums in the layout the combine kernel reads.  A consumer warp
// whose wait times out keeps taking the barriers without touching the stage,
// so that no warp waits on it; every wait is bounded.
#pragma once

#include <cuda_fp16.h>

#include "stream.cuh"

namespace mtf {

template <int NC>
struct StreamTC {
  static constexpr int NT = (NC + 1) / 2;            // n8 tiles (4 real columns per right-hand side)
  static constexpr int K = StreamK<NC, 3>::K;        // partial sums per row piece, as in stream.cuh
  static constexpr int L = st_piece_len<3>();        // complex entries per piece
  static constexpr int LC = (L + 7) / 8 * 8;         // entries copied per row slot
  static constexpr int RBP = (LC * 4 + 127) / 128 * 128 + 16;  // row slot: the largest tiled pitch
  static constexpr int XB = (L + 2) * 8 + 16;        // input slice slot (padded: slices 8 banks apart)
  static constexpr int ROWS = 16;
  static constexpr int SB = ((ROWS * RBP + 2 * NC * XB) + 127) / 128 * 128;
  static constexpr int RED = 2 * NT * 8 * 32 * 16;   // two buffers of 8 warps x 32 lanes x float4 per tile
  static constexpr int S0 = (kStSmemBudget - RED) / SB;
  static constexpr int S = S0 < kStMaxStages ? S0 : kStMaxStages;
  static constexpr size_t smem = size_t(S) * SB + RED + size_t(S) * (2 * sizeof(uint64_t) + sizeof(int4));
  static_assert(S >= 2, "the stage ring needs at least two stages");
  static_assert(smem <= 232448, "shared memory above the per-CTA limit");
  static_assert(st_unit_rows<3>() == ROWS && st_consumers<3>() == 8, "units of 16 rows, 8 consumer warps");
};

__device__ __forceinline__ uint32_t tc_pack(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int NC>
__global__ void __launch_bounds__(9 * 32, 1) k_stream_tc(const void* __restrict__ tiled,
                                                        const int4* __restrict__ units,
                                                        const int64_t* __restrict__ toff, int n_units, int pmax,
                                                        const float* __restrict__ x32, int64_t ld32, int c0,
                                                        float* __restrict__ part, unsigned* __restrict__ err) {
  using TC = StreamTC<NC>;
  constexpr int S = TC::S, SB = TC::SB, RBP = TC::RBP, XB = TC::XB, ROWS = TC::ROWS, NT = TC::NT, K = TC::K;
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  extern __shared__ __align__(128) unsigned char smem[];
  float* red = reinterpret_cast<float*>(smem + size_t(S) * SB);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(S) * SB + TC::RED);
  uint64_t* empty = full + S;
  int4* meta = reinterpret_cast<int4*>(empty + S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 8);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == 8) {
    // producer: one lane issues every copy
    if (lane != 0) return;
    const unsigned char* ent = static_cast<const unsigned char*>(tiled);
    const uint64_t stream_pol = l2_policy_evict_first();
    int k = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++k) {
      const int4 rec = units[u];
      const int64_t src = toff[u];
      const int s = k % S;
      if (!mbar_wait_bounded(&empty[s], (uint32_t(k / S) & 1u) ^ 1u, kStWaitNs)) {
        atomicExch(err, 1u);
        return;
      }
      const int N = rec.x, len = rec.w & 0xfff, nrows = (rec.w >> 24) & 0xff;
      const uint32_t rows_bytes = uint32_t(nrows * st_tile_pitch(4, len));  // the unit's contiguous run
      uint32_t total = rows_bytes;
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
      bulk_g2s_hint(st, ent + src, rows_bytes, &full[s], stream_pol);
#pragma unroll
      for (int q = 0; q < 2 * NC; ++q) bulk_g2s(st + ROWS * RBP + q * XB, x32 + 2 * xa[q], xbytes[q], &full[s]);
    }
    return;
  }

  const int tid = threadIdx.x;  // consumer thread 0 .. 255
  bool dead = false;
  int k = 0, rbuf = 0;
  for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++k) {
    const int s = k % S;
    if (!dead && !mbar_wait_bounded(&full[s], uint32_t(k / S) & 1u, kStWaitNs)) {
      dead = true;
      if (lane == 0) atomicExch(err, 1u);
    }
    float acc[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    int4 rec = make_int4(0, 0, 0, 0);
    if (!dead) {
      rec = meta[s];
      const int N = rec.x, len = rec.w & 0xfff;
      const unsigned char* st = smem + size_t(s) * SB;
      // ldmatrix x4: lanes 0-7 rows 0-7 (k 0-7), 8-15 rows 8-15 (k 0-7),
      // 16-23 rows 0-7 (k 8-15), 24-31 rows 8-15 (k 8-15)
      const int pitch = st_tile_pitch(4, len);
      const uint32_t abase = smem_u32(st) + uint32_t(((lane & 7) + ((lane >> 3) & 1) * 8) * pitch + (lane >> 4) * 16);
      const int n = lane >> 2, tig = lane & 3, p = n & 1;
      // this lane's input column per tile: slice q = 4 t + n / 2 (the slice
      // starts one entry early when its first entry is odd; ld32 is even)
      const float2* xq[NT];
      bool qok[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int q = t * 4 + (n >> 1);
        qok[t] = q < 2 * NC;
        xq[t] = reinterpret_cast<const float2*>(st + ROWS * RBP + q * XB) + ((rec.z + (q & 1) * N) & 1);
      }
      const int nch = (len + 7) >> 3;
      for (int ch = warp; ch < nch; ch += 8) {
        uint32_t a0, a1, a2, a3;
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                     : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                     : "r"(abase + uint32_t(ch) * 32u));
        const int cb = ch * 8 + tig;  // complex column of b0; b1 at cb + 4
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          float2 v0 = make_float2(0.f, 0.f), v1 = v0;
          if (qok[t]) {
            if (cb < len) v0 = xq[t][cb];
            if (cb + 4 < len) v1 = xq[t][cb + 4];
          }
          // real-part column: (x_re, -x_im); imaginary-part column: (x_im, x_re)
          const uint32_t b0 = p ? tc_pack(v0.y, v0.x) : tc_pack(v0.x, -v0.y);
          const uint32_t b1 = p ? tc_pack(v1.y, v1.x) : tc_pack(v1.x, -v1.y);
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
              "{%0, %1, %2, %3};"
              : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
              : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
      }
    }
    float* rb = red + size_t(rbuf) * NT * 8 * 32 * 4;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      reinterpret_cast<float4*>(rb)[(t * 8 + warp) * 32 + lane] = make_float4(acc[t][0], acc[t][1], acc[t][2], acc[t][3]);
    // release the stage: order this warp's shared reads before the next bulk write
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0 && !dead) mbar_arrive(&empty[s]);
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (!dead) {
      const int nrows = (rec.w >> 24) & 0xff, piece = (rec.w >> 12) & 0xfff;
      // C fragment of lane l: (row l/4, columns 2 (l%4) + {0, 1}) and row l/4 + 8
      for (int idx = tid; idx < NT * 128; idx += 256) {
        const int t = idx >> 7, l = (idx >> 2) & 31, j = idx & 3;
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += rb[((t * 8 + w) * 32 + l) * 4 + j];
        const int row = (l >> 2) + (j >> 1) * 8, v = t * 8 + (l & 3) * 2 + (j & 1);
        if (row < nrows && v < 4 * NC) part[(int64_t(rec.y + row) * pmax + piece) * K + v] = sum;
      }
    }
    rbuf ^= 1;
  }
}

// one launch of the tensor-core stream for right-hand sides c0 .. c0+NC-1
template <int NC>
void launch_stream_tc(mtf_system sys, const void* tiled, const StreamUnits& su, const float* x32, int64_t ld32,
                      int c0, float* part, int kid, cudaStream_t s) {
  using TC = StreamTC<NC>;
  MTF_REQUIRE(ld32 % 2 == 0 && (reinterpret_cast<uintptr_t>(x32) & 15) == 0 &&
                  (reinterpret_cast<uintptr_t>(tiled) & 15) == 0,
              MTF_ERR_ARG, "streamed vectors and operators must be 16-byte aligned with an even column stride");
  auto kfn = k_stream_tc<NC>;
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load(std::memory_order_relaxed) & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TC::smem)));
    opted.fetch_or(bit);
  }
  MTF_LAUNCH(kid, s,
             launch_pdl(kfn, dim3(unsigned(sys->mv_grid)), dim3(9 * 32), TC::smem, s, tiled, su.d_units.p,
                        su.d_toff.p, int(su.n_units), su.pmax, x32, ld32, c0, part, sys->d_mv_ctl.p + 2));
}

}  // namespace mtf
