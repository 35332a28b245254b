// Bulk-copy streaming matvec of the FP32-stored MTF operator (Eq. 16 applied
// as y = 2 A x + X x, block by block, as in the FP64 kernel).
//
// The dense blocks are cut into work units: a unit is one row piece of at
// most kMvUnit entries (row m of block i, columns [c, c + len)), every row of
// block i in P_i pieces of near-equal length.  Units are ordered piece-major
// within a block (all rows of piece 0, then piece 1, ...), and warp g of the
// grid takes units g, g + W, g + 2W, ... (W warps), so the warps of one SM
// work on neighbouring rows of the same column piece and share its slice of
// the input vector in L1.  Each warp owns a private ring of S shared-memory
// stages; one lane fetches units with the TMA engine (cp.async.bulk, one
// mbarrier per stage) S units ahead of the one the warp consumes, with the
// unit records themselves prefetched one unit further ahead, so nothing on
// a warp's path waits on a global round trip except the matrix data itself.
//
// A unit's partial sums (8 per right-hand side: T and K against the D and N
// slots) are reduced over the warp and stored; k_mv_combine then adds each
// row's pieces in fixed order (the result does not depend on the schedule)
// and applies the epilogue: rho coupling, factor 2 and the exchange rows X x.
//
// A wait on a bulk copy that does not complete within ~0.5 s sets an error
// word instead of hanging; the host reports it as MTF_ERR_TIMEOUT.
#include <algorithm>

#include "bulk.h"
#include "common.h"

namespace mtf {

constexpr int kMvWarps = 8;
constexpr int kMvUnit = 512;    // float4 entries (8 KB) per unit
constexpr int kMvStages = 3;
constexpr uint64_t kMvWaitNs = 500000000ull;

template <int NC>
struct MvK {
  static constexpr int K = NC == 1 ? 8 : (NC == 2 ? 16 : 32);  // partial sums per unit, padded to 2^k
  static constexpr int SH = NC == 1 ? 2 : (NC == 2 ? 1 : 0);  // value index = lane >> SH
};

// unit record: N of the block, global row, first input column (dof offset of
// the block + first column of the piece), len | piece << 12; plus the float4
// offset of the piece in the stored blocks
template <int NC>
__global__ void __launch_bounds__(kMvWarps * 32, 1) k_matvec_bulk(const float4* __restrict__ TK,
                                                                   const int4* __restrict__ units,
                                                                   const int64_t* __restrict__ usrc, int n_units,
                                                                   int pmax, const float* __restrict__ x32,
                                                                   int64_t ld32, int c0, float* __restrict__ part,
                                                                   unsigned* __restrict__ err) {
  constexpr int K = MvK<NC>::K, SH = MvK<NC>::SH, S = kMvStages;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* tail = smem_raw + size_t(kMvWarps) * S * kMvUnit * sizeof(float4);
  float4* ring = reinterpret_cast<float4*>(smem_raw) + size_t(warp) * S * kMvUnit;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tail) + warp * S;
  int4* meta = reinterpret_cast<int4*>(tail + size_t(kMvWarps) * S * sizeof(uint64_t)) + warp * S;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  const int W = int(gridDim.x) * kMvWarps;
  int u_next = int(blockIdx.x) * kMvWarps + warp;  // next unit to issue
  int issued = 0, consumed = 0;
  int4 nrec = make_int4(0, 0, 0, 0);  // lane 0: record of u_next, loaded one issue ahead
  int64_t nsrc = 0;
  if (lane == 0 && u_next < n_units) {
    nrec = units[u_next];
    nsrc = usrc[u_next];
  }
  auto issue = [&]() {
    if (lane == 0) {
      const int s = issued % S;
      meta[s] = nrec;
      const uint32_t bytes = uint32_t(nrec.w & 0xfff) * uint32_t(sizeof(float4));
      mbar_arrive_expect_tx(&bar[s], bytes);
      bulk_g2s(ring + size_t(s) * kMvUnit, TK + nsrc, bytes, &bar[s]);
      const int un = u_next + W;
      if (un < n_units) {
        nrec = units[un];
        nsrc = usrc[un];
      }
    }
    u_next += W;
    ++issued;
  };

  for (int k = 0; k < S && u_next < n_units; ++k) issue();
  const float2* x2 = reinterpret_cast<const float2*>(x32);
  while (consumed < issued) {
    const int s = consumed % S;
    if (!mbar_wait_bounded(&bar[s], uint32_t(consumed / S) & 1u, kMvWaitNs)) {
      if (lane == 0) atomicExch(err, 1u);
      // let the other copies of this warp land (bounded) before leaving
      for (int q = consumed + 1; q < issued; ++q) mbar_wait_bounded(&bar[q % S], uint32_t(q / S) & 1u, kMvWaitNs);
      return;
    }
    const int4 info = meta[s];
    const int N = info.x, row = info.y, len = info.w & 0xfff, p = info.w >> 12;
    const float2* xb = x2 + info.z;
    float v[K];
#pragma unroll
    for (int q = 0; q < K; ++q) v[q] = 0.f;
    const float4* st = ring + size_t(s) * kMvUnit;
#pragma unroll 4
    for (int e = lane; e < len; e += 32) {
      const float4 a = st[e];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 xd = __ldg(xb + (c0 + c) * ld32 + e);
        const float2 xn = __ldg(xb + (c0 + c) * ld32 + e + N);
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
    }
    // stage s has been read: refill it while this unit is reduced
    fence_proxy_async_smem();
    __syncwarp();
    ++consumed;
    if (u_next < n_units) issue();
    WarpTransposeSum<K>::run(v, lane, 16);
    if ((lane & ((1 << SH) - 1)) == 0) part[(int64_t(row) * pmax + p) * K + (lane >> SH)] = v[0];
  }
}

// y rows of one block row m (one warp per global row): sum the row's P piece
// partials in order, then 2 (K x_D + rho^-1 T x_N) + X_D x and
// 2 (-rho T x_D + K x_N) + X_N x per right-hand side (lane c < NC).  The
// epilogue runs in the output precision: FP32 (rho, 1/rho and the exchange
// values from their FP32 copies) for FP32 output, FP64 otherwise.  FP64
// arithmetic is kept off the FP32 path on purpose: the FP64 pipe is narrow
// enough that a few dozen FP64 instructions per row dominate this kernel.
template <int NC, class XT, class YT>
__global__ void __launch_bounds__(256) k_mv_combine(
    const float* __restrict__ part, int pmax, const int32_t* __restrict__ row_blk, const int32_t* __restrict__ blk_N,
    const int64_t* __restrict__ blk_dof_off, const int64_t* __restrict__ blk_row_off, const XEntry* __restrict__ xe,
    const double* __restrict__ xval, const float* __restrict__ xval32, const double* __restrict__ rho,
    const float* __restrict__ rho32, const XT* __restrict__ x, int64_t ldx, YT* __restrict__ y, int64_t ldy, int c0,
    int64_t n_rows) {
  constexpr int K = MvK<NC>::K;
  using AT = YT;
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int i = row_blk[row];
  const int N = blk_N[i];
  const int P = max(1, (N + kMvUnit - 1) / kMvUnit);
  float tot = 0.f;
  if (lane < K)
    for (int p = 0; p < P; ++p) tot += part[(row * pmax + p) * K + lane];
  float a[8];
  const int cl = lane < NC ? lane : 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = __shfl_sync(0xffffffffu, tot, cl * 8 + q);
  if (lane >= NC) return;
  const int64_t m = row - blk_row_off[i];
  const int64_t off = blk_dof_off[i];
  AT rr, ri, ir, ii;
  if constexpr (sizeof(AT) == 4) {
    rr = rho32[4 * i];
    ri = rho32[4 * i + 1];
    ir = rho32[4 * i + 2];
    ii = rho32[4 * i + 3];
  } else {
    rr = rho[2 * i];
    ri = rho[2 * i + 1];
    const AT rn = rr * rr + ri * ri;
    ir = rr / rn;
    ii = -ri / rn;
  }
  const int col = c0 + lane;
  const XT* xc = x + 2 * int64_t(col) * ldx;
  AT yDr = AT(2) * (AT(a[4]) + (AT(a[2]) * ir - AT(a[3]) * ii));
  AT yDi = AT(2) * (AT(a[5]) + (AT(a[2]) * ii + AT(a[3]) * ir));
  AT yNr = AT(2) * (AT(a[6]) - (AT(a[0]) * rr - AT(a[1]) * ri));
  AT yNi = AT(2) * (AT(a[7]) - (AT(a[0]) * ri + AT(a[1]) * rr));
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const XEntry X = xe[6 * row + e];
    AT xv;
    if constexpr (sizeof(AT) == 4) xv = xval32[6 * row + e];
    else xv = xval[6 * row + e];
    const int Nj = X.ab >> 4;
    yDr += xv * AT(xc[2 * int64_t(X.col)]);
    yDi += xv * AT(xc[2 * int64_t(X.col) + 1]);
    yNr += xv * AT(xc[2 * (int64_t(X.col) + Nj)]);
    yNi += xv * AT(xc[2 * (int64_t(X.col) + Nj) + 1]);
  }
  YT* yc = y + 2 * (int64_t(col) * ldy + off);
  yc[2 * m] = yDr;
  yc[2 * m + 1] = yDi;
  yc[2 * (N + m)] = yNr;
  yc[2 * (N + m) + 1] = yNi;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void build_units(mtf_mesh m, cudaStream_t s) {
  if (m->mv_units_ready) return;
  std::vector<int4> u;
  std::vector<int64_t> src;
  int pmax = 1;
  for (int i = 0; i < m->nd; ++i) {
    const int N = m->blk[i].N;
    const int P = std::max(1, (N + kMvUnit - 1) / kMvUnit);
    const int ps = (N + P - 1) / P;
    MTF_REQUIRE(ps <= kMvUnit, MTF_ERR_MESH, "matvec piece longer than a stage");
    pmax = std::max(pmax, P);
    for (int p = 0; p < P; ++p)
      for (int r = 0; r < N; ++r) {
        const int c = p * ps, len = std::min(ps, N - c);
        MTF_REQUIRE(len > 0, MTF_ERR_MESH, "empty matvec piece");
        u.push_back(make_int4(N, int(m->blk[i].row_off + r), int(m->blk[i].dof_off + c), len | (p << 12)));
        src.push_back(m->blk[i].mat_off + int64_t(r) * N + c);
      }
  }
  MTF_REQUIRE(m->n_total < (int64_t(1) << 31) && int64_t(u.size()) < (int64_t(1) << 31), MTF_ERR_MESH,
              "mesh too large for the streaming matvec tables");
  m->mv_n_units = int64_t(u.size());
  m->mv_pmax = pmax;
  m->d_mv_units.alloc(u.size());
  m->d_mv_src.alloc(src.size());
  if (!u.empty()) {
    MTF_CUDA(cudaMemcpyAsync(m->d_mv_units.p, u.data(), u.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    MTF_CUDA(cudaMemcpyAsync(m->d_mv_src.p, src.data(), src.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MTF_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  }
  m->mv_units_ready = true;
}

static void ensure_mv_scratch(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  build_units(m, s);
  const size_t npart = size_t(m->n_rows) * m->mv_pmax * 32;
  if (sys->d_mv_part.n != npart) {
    sys->d_mv_part.alloc(npart);
    sys->d_mv_ctl.alloc(4);
    MTF_CUDA(cudaMemsetAsync(sys->d_mv_ctl.p, 0, 4 * sizeof(unsigned), s));
  }
  if (!sys->mv_grid) {
    int dev = 0, sms = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    MTF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    sys->mv_grid = std::max(1, sms);
  }
}

static constexpr size_t mv_smem() {
  return size_t(kMvWarps) * kMvStages * (kMvUnit * sizeof(float4) + sizeof(uint64_t) + sizeof(int4));
}

template <int NC, class XT, class YT>
static void mv_launch(mtf_system sys, const XT* x, int64_t ldx, const float* x32, int64_t ld32, YT* y, int64_t ldy,
                      int c0, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  auto kfn = k_matvec_bulk<NC>;
  MTF_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(mv_smem())));
  MTF_LAUNCH(KID_MATVEC32, s, kfn<<<unsigned(sys->mv_grid), kMvWarps * 32, mv_smem(), s>>>(
      reinterpret_cast<const float4*>(sys->d_TK32.p), m->d_mv_units.p, m->d_mv_src.p, int(m->mv_n_units),
      m->mv_pmax, x32, ld32, c0, sys->d_mv_part.p, sys->d_mv_ctl.p + 2));
  MTF_LAUNCH(KID_MVCOMBINE, s, k_mv_combine<NC, XT, YT><<<unsigned((m->n_rows * 32 + 255) / 256), 256, 0, s>>>(
      sys->d_mv_part.p, m->mv_pmax, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p, m->d_blk_row_off.p,
      m->d_xent.p, sys->d_xval.p, sys->d_xval32.p, sys->d_rho.p, sys->d_rho32.p, x, ldx, y, ldy, c0, m->n_rows));
}

template <class XT, class YT>
static void mv_all(mtf_system sys, const XT* x, int64_t ldx, const float* x32, int64_t ld32, YT* y, int64_t ldy,
                   int nrhs, cudaStream_t s) {
  ensure_mv_scratch(sys, s);
  for (int c0 = 0; c0 < nrhs; c0 += 4) {
    const int nc = std::min(4, nrhs - c0);
    if (nc == 1) mv_launch<1>(sys, x, ldx, x32, ld32, y, ldy, c0, s);
    else if (nc == 2) mv_launch<2>(sys, x, ldx, x32, ld32, y, ldy, c0, s);
    else if (nc == 3) mv_launch<3>(sys, x, ldx, x32, ld32, y, ldy, c0, s);
    else mv_launch<4>(sys, x, ldx, x32, ld32, y, ldy, c0, s);
  }
}

void launch_matvec_stream64(mtf_system sys, const double* x, int64_t ldx, const float* x32, int64_t ld32, double* y,
                            int64_t ldy, int nrhs, cudaStream_t s) {
  mv_all<double, double>(sys, x, ldx, x32, ld32, y, ldy, nrhs, s);
}

void launch_matvec_f32(mtf_system sys, const float* x, int64_t ldx, float* y, int64_t ldy, int nrhs,
                       cudaStream_t s) {
  mv_all<float, float>(sys, x, ldx, x, ldx, y, ldy, nrhs, s);
}

// Throws MTF_ERR_TIMEOUT if a launch of the streaming matvec gave up on a
// bulk copy since the last check (synchronises the stream) and clears the
// error word.
void check_matvec_stream(mtf_system sys, cudaStream_t s) {
  if (!sys->d_mv_ctl.p) return;
  unsigned ctl[4];
  MTF_CUDA(cudaMemcpyAsync(ctl, sys->d_mv_ctl.p, sizeof(ctl), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  if (ctl[2] == 0) return;
  MTF_CUDA(cudaMemsetAsync(sys->d_mv_ctl.p, 0, 4 * sizeof(unsigned), s));
  MTF_CUDA(cudaStreamSynchronize(s));
  throw Error{MTF_ERR_TIMEOUT, "a bulk copy of the streaming matvec did not complete in time"};
}

}  // namespace mtf
