// Streaming tensor-core product with one operator: for every work unit
// u = {a_base, b_base, kc0, kc1} the chunks kc0 <= kc < kc1 pair operator
// tile a_base + kc with input chunk b_base + kc, and
//   D = sum_kc A_kc B_kc^T
// is accumulated in TMEM (M = 128 rows x NB columns, FP32) from FP16 parts:
//   NPA = 1 (the operator is one FP16 value):  A Bhi + A Blo
//   NPA = 2 (FP16 hi + lo of the operator):     Ahi Bhi + Ahi Blo + Alo Bhi
// Both operands are K-major tiles of 64 FP16 per row in the 128-byte swizzle,
// loaded by one cp.async.bulk.tensor.4d copy each (tc.cuh, tc_plan.h).
// The pipeline is the tensor-core matvec's: warp 0 lane 0 produces into a
// ring of stages, warp 1 allocates TMEM and one lane issues the MMAs and
// commits, warps 2-5 drain finished TMEM buffers (two, so that a unit's
// epilogue overlaps the next unit's MMAs).  Units are taken round-robin, or
// from a schedule (sched[sched_off[b] .. sched_off[b + 1]) for CTA b).
// Epilogues:
//   EPI 0: raw row sums to part[(u * 128 + row) * NB + col]
//   EPI 1: W_c[128 u + row] -= (D[row][2c] + i D[row][2c + 1]) * s_c,
//          s_c = inv_scale(colmax[c]) / 2^14, for c < ncols, rows < n_limit
//          (the Gram-Schmidt update of W against a basis stored x 2^14).
//   EPI 2: the block-OSRC formation (tc_plan.h, plan_tt): unit u covers rows
//          r = info.y + row and complex columns c = info.z + col / 2 of the
//          symmetric T~ of block info.x; (D[row][2j], D[row][2j + 1]) * inv
//          goes to T~(r, c) when c >= r and to T~(c, r) when c > r.
// Every wait is bounded (0.5 s) and ends in the error word.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "tc.cuh"
#include "tc_plan.h"

namespace mtf {

template <int NPA, int NB>
struct TcsCfg {
  static constexpr int SA = NPA * kTcRows * 128;
  static constexpr int SBB = 2 * NB * 128;
  static constexpr int SB = SA + SBB;
  static constexpr int S0 = (220 * 1024) / SB;
  static constexpr int S = S0 > 6 ? 6 : S0;  // up to 6 stages (about 100 KB of operator tiles in flight)
  static constexpr uint32_t TMEM = 2 * NB < 32 ? 32 : 2 * NB;  // two buffers of NB columns
  static constexpr size_t smem = size_t(S) * SB + 1024 + 256;
  static_assert(S >= 2 && smem <= 232448 && SB % 1024 == 0, "stage ring");
};

constexpr uint64_t kTcsWaitNs = 500000000ull;

// Work units given by a rule instead of a list (no host staging, so launches
// can be queued ahead of the host):
//   kind 0: units[u] (explicit list), output index u
//   kind 1: u = g P + p -> {g a, 0, p b, min(a, (p + 1) b)}: a = chunks per
//           row tile, P = c pieces of b chunks (the Gram-Schmidt dots)
//   kind 2: u = e -> {e a, 0, 0, b}: a = chunks per row tile, b chunks used
//           (the Gram-Schmidt update), output index e
struct TcUnits {
  int kind = 0;
  int a = 0, b = 0, c = 0;
  const int4* list = nullptr;
  __device__ __forceinline__ int4 get(int u) const {
    if (kind == 1) {
      const int g = u / c, p = u % c;
      return make_int4(g * a, 0, p * b, min(a, (p + 1) * b));
    }
    if (kind == 2) return make_int4(u * a, 0, 0, b);
    return list[u];
  }
};

// outputs of the block-OSRC formation (EPI 2)
struct TcTtOut {
  const int4* info = nullptr;    // per unit {block, first row, first complex column, 0}
  const int* N = nullptr;        // per block: order of T~
  const int* ldt = nullptr;      // per block: row stride of T~ (complex entries)
  const int64_t* off = nullptr;  // per block: first complex entry of T~
  const float* inv = nullptr;    // per block: 1 / (operand scales)
  float2* T = nullptr;
};

__device__ __forceinline__ float tcs_inv_scale(unsigned bits) {
  const float a = __uint_as_float(bits);
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, ex - 14);
}

template <int NPA, int NB, int EPI>
__global__ void __launch_bounds__(192, 1) k_tc_stream(const __grid_constant__ CUtensorMap amap,
                                                      const __grid_constant__ CUtensorMap bmap, const TcUnits units,
                                                      int n_units, const int* __restrict__ sched,
                                                      const int* __restrict__ sched_off, float* __restrict__ part,
                                                      float* __restrict__ W, int64_t ldw, int ncols, int64_t n_limit,
                                                      const unsigned* __restrict__ colmax, unsigned* __restrict__ err,
                                                      const TcTtOut tt) {
  using C = TcsCfg<NPA, NB>;
  constexpr int S = C::S, SB = C::SB, SA = C::SA;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(S) * SB);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this CTA's units: u = unit(q) for q in [q0, q1) with stride qs
  const bool listed = sched != nullptr;
  const int q0 = listed ? sched_off[blockIdx.x] : int(blockIdx.x);
  const int q1 = listed ? sched_off[blockIdx.x + 1] : n_units;
  const int qs = listed ? 1 : int(gridDim.x);
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
      for (int q = q0; q < q1 && ok; q += qs) {
        const int4 U = units.get(listed ? sched[q] : q);
        for (int kc = U.z; kc < U.w; ++kc, ++k) {
          const int st = k % S;
          if (!mbar_wait_bounded(&empty[st], (uint32_t(k / S) & 1u) ^ 1u, kTcsWaitNs)) {
            atomicExch(err, 1u);
            ok = false;
            break;
          }
          unsigned char* sa = smem + size_t(st) * SB;
          mbar_arrive_expect_tx(&full[st], uint32_t(SB));
          tma_load_4d(sa, &amap, 0, 0, 0, U.x + kc, &full[st], pol_a);
          tma_load_4d(sa + SA, &bmap, 0, 0, 0, U.y + kc, &full[st], pol_b);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16_m128(NB);
      int k = 0, ub = 0;
      bool ok = true;
      for (int q = q0; q < q1 && ok; q += qs, ++ub) {
        const int4 U = units.get(listed ? sched[q] : q);
        const int buf = ub & 1;
        if (!mbar_wait_bounded(&tempty[buf], (uint32_t(ub >> 1) & 1u) ^ 1u, kTcsWaitNs)) {
          atomicExch(err, 1u);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + uint32_t(buf * NB);
        for (int kc = U.z; kc < U.w; ++kc, ++k) {
          const int st = k % S;
          if (!mbar_wait_bounded(&full[st], uint32_t(k / S) & 1u, kTcsWaitNs)) {
            atomicExch(err, 1u);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + size_t(st) * SB), sb = sa + SA;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ah = sw128_desc(sa + kk * 32);
            const uint64_t bh = sw128_desc(sb + kk * 32), bl = sw128_desc(sb + NB * 128 + kk * 32);
            const uint32_t acc = (kc != U.z || kk != 0) ? 1u : 0u;
            tc_mma_f16(d, ah, bh, idesc, acc);
            tc_mma_f16(d, ah, bl, idesc, 1u);
            if constexpr (NPA == 2) tc_mma_f16(d, sw128_desc(sa + 16384 + kk * 32), bh, idesc, 1u);
          }
          tc_commit(&empty[st]);
        }
        if (ok) tc_commit(&tfull[buf]);
      }
    }
  } else {
    const int quarter = warp & 3;
    const int row = 32 * quarter + lane;
    int ub = 0;
    for (int q = q0; q < q1; q += qs, ++ub) {
      const int u = listed ? sched[q] : q;
      const int buf = ub & 1;
      if (!mbar_wait_bounded(&tfull[buf], uint32_t(ub >> 1) & 1u, kTcsWaitNs)) {
        if (lane == 0) atomicExch(err, 1u);
        break;
      }
      tc_fence_after();
      const uint32_t ta = tmem + (uint32_t(32 * quarter) << 16) + uint32_t(buf * NB);
      if constexpr (EPI == 0) {
        float* dst = part + (size_t(u) * kTcRows + row) * NB;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
          float v[16];
          tmem_ld16(ta + uint32_t(c0), v);
          float4* d4 = reinterpret_cast<float4*>(dst + c0);
          d4[0] = make_float4(v[0], v[1], v[2], v[3]);
          d4[1] = make_float4(v[4], v[5], v[6], v[7]);
          d4[2] = make_float4(v[8], v[9], v[10], v[11]);
          d4[3] = make_float4(v[12], v[13], v[14], v[15]);
        }
      } else if constexpr (EPI == 2) {
        const int4 I = tt.info[u];
        const int n = tt.N[I.x], ld = tt.ldt[I.x];
        const int64_t off = tt.off[I.x];
        const float inv = tt.inv[I.x];
        const int r = I.y + row;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
          float v[16];
          tmem_ld16(ta + uint32_t(c0), v);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = I.z + c0 / 2 + i;
            if (r < n && c < n && c >= r) {
              const float2 o = make_float2(v[2 * i] * inv, v[2 * i + 1] * inv);
              tt.T[off + int64_t(r) * ld + c] = o;
              if (c > r) tt.T[off + int64_t(c) * ld + r] = o;
            }
          }
        }
      } else {
        const int64_t kk = int64_t(u) * kTcRows + row;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
          float v[16];
          tmem_ld16(ta + uint32_t(c0), v);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = c0 / 2 + i;
            if (c < ncols && kk < n_limit) {
              const float sc = tcs_inv_scale(colmax[c]) * (1.f / 16384.f);
              float2* wp = reinterpret_cast<float2*>(W + 2 * (int64_t(c) * ldw + kk));
              float2 o = *wp;
              o.x -= v[2 * i] * sc;
              o.y -= v[2 * i + 1] * sc;
              *wp = o;
            }
          }
        }
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

}  // namespace mtf
