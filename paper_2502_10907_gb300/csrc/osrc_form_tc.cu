// Formation of the block-OSRC operators T~_i = W_i diag(f_i) W_i^T (Sec. 4.4,
// Eq. 19) on the fifth-generation tensor cores, once per assembly: W_i (the
// mode basis, a mesh constant) and f_i (the symbol, which depends on k_i).
//
// Formulation and layout: tc_plan.h (plan_tt).  Both operands are split into
// FP16 hi + lo after a power-of-two scaling per block (W by s_A, the scaled
// modes f^(t) W by s_B, so that every entry is below 2^14), and the three
// products hi*hi + hi*lo + lo*hi are summed in FP32 by k_tc_stream<2, 128, 2>
// (tc_stream.cuh), whose epilogue writes the interleaved complex rows of T~
// (FP32) and their mirror images.  The A tiles of W are built once per
// system; per formation only the scales and the B chunks of the scaled modes
// are rebuilt.  Entry error about 2^-21 of the block's largest |W|^2 |f|
// times sqrt(N_i); T~ only steers the Krylov iteration (the flexible GMRES
// uses the vectors it applied), it does not enter the solution.
#include <cuda.h>
#include <cuda_fp16.h>

#include <atomic>

#include "common.h"
#include "tc.cuh"
#include "tc_plan.h"
#include "tc_stream.cuh"

namespace mtf {

void tc_encode_map(void* map, const void* base, int rows, int parts, int64_t count);
void stream_prepare(mtf_system sys, cudaStream_t s);
void check_matvec_stream(mtf_system sys, cudaStream_t s);

struct TtForm {
  TtPlan plan;
  bool a_built = false;
  int n_cta = 0;
  DevBuf<__half> A, B;             // A tiles of W, B chunks of the scaled modes
  DevBuf<int4> a_info, b_info;     // A tile {blk, mt, kc, 0}; B chunk {blk, nt, kc, 0}
  DevBuf<int4> units, info;        // unit {a tile, b chunk, 0, n_kc}; {blk, row0, col0, 0}
  DevBuf<int> N, ldt;
  DevBuf<int64_t> off, vt_off, row_off;
  DevBuf<float> wmax, scale, inv;  // per mode: max_r |W(r, j)|; per block: (s_A, s_B); 1 / (s_A s_B)
  CUtensorMap amap{}, bmap{};
};

void destroy_tt(TtForm* t) { delete t; }

// power-of-two s with a s < 2^14 (1 for a = 0)
__device__ __forceinline__ float tt_pow2_scale(float a) {
  if (!(a > 0.f)) return 1.f;
  int ex;
  frexpf(a, &ex);
  return ldexpf(1.f, 14 - ex);
}

// largest |W(r, j)| over the dofs r of mode j (one warp per mode); W is
// stored as rows j of length ld (the RWG dofs contiguous)
__global__ void k_tt_wmax(const float* __restrict__ Vt, const int64_t* __restrict__ vt_off,
                          const int32_t* __restrict__ row_blk, const int64_t* __restrict__ row_off,
                          const int* __restrict__ Nb, int64_t n_rows, float* __restrict__ wmax) {
  const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= n_rows) return;
  const int i = row_blk[q];
  const int N = Nb[i], ld = (N + 3) & ~3;
  const int64_t j = q - row_off[i];
  const float* w = Vt + vt_off[i] + j * ld;
  float m = 0.f;
  for (int r = lane; r < N; r += 32) m = fmaxf(m, fabsf(w[r]));
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) wmax[q] = m;
}

// per block (one CTA each): s_A from max |W|, s_B from max |f^(t)_j| wmax_j
__global__ void k_tt_scales(const float* __restrict__ wmax, const float2* __restrict__ f,
                            const int64_t* __restrict__ row_off, const int* __restrict__ Nb,
                            float* __restrict__ scale, float* __restrict__ inv) {
  const int i = blockIdx.x;
  const int N = Nb[i];
  const int64_t r0 = row_off[i];
  float ma = 0.f, mb = 0.f;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const float w = wmax[r0 + j];
    const float2 fj = f[r0 + j];
    ma = fmaxf(ma, w);
    mb = fmaxf(mb, fmaxf(fabsf(fj.x), fabsf(fj.y)) * w);
  }
  __shared__ float sa[32], sb[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = ma;
    sb[threadIdx.x >> 5] = mb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < int(blockDim.x >> 5); ++w) {
      ma = fmaxf(ma, sa[w]);
      mb = fmaxf(mb, sb[w]);
    }
    const float a = tt_pow2_scale(ma), b = tt_pow2_scale(mb);
    scale[2 * i] = a;
    scale[2 * i + 1] = b;
    inv[i] = 1.f / (a * b);  // powers of two: exact
  }
}

__device__ __forceinline__ void tt_split8(const float* x, __half* hi, __half* lo) {
  __align__(16) __half h[8], l[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    h[e] = __float2half_rn(x[e]);
    l[e] = __float2half_rn(x[e] - __half2float(h[e]));
  }
  *reinterpret_cast<uint4*>(hi) = *reinterpret_cast<const uint4*>(h);
  *reinterpret_cast<uint4*>(lo) = *reinterpret_cast<const uint4*>(l);
}

// A tiles: thread (tile, 8-mode group g, row rho) packs W(r, 64 kc + 8 g + e)
// * s_A, r = 128 mt + rho, e < 8 (zero past N); consecutive threads take
// consecutive rows, so every mode's read is coalesced
__global__ void k_tt_tile_a(const float* __restrict__ Vt, const int64_t* __restrict__ vt_off,
                            const int4* __restrict__ a_info, const int* __restrict__ Nb,
                            const float* __restrict__ scale, int64_t n_tiles, __half* __restrict__ A) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_tiles * 8 * kTcRows) return;
  const int rho = int(t % kTcRows), g = int((t / kTcRows) % 8);
  const int64_t tile = t / (8 * kTcRows);
  const int4 I = a_info[tile];
  const int N = Nb[I.x], ld = (N + 3) & ~3;
  const int r = I.y * kTcRows + rho;
  const float sa = scale[2 * I.x];
  const float* w = Vt + vt_off[I.x];
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int j = I.z * 64 + 8 * g + e;
    x[e] = (r < N && j < N) ? w[int64_t(j) * ld + r] * sa : 0.f;
  }
  tt_split8(x, A + tc_tile_index(tile, 2, 0, rho, 8 * g), A + tc_tile_index(tile, 2, 1, rho, 8 * g));
}

// B chunks: row gamma of chunk (blk, nt, kc) is f^(gamma & 1)_j W(c, j) * s_B
// with c = 64 nt + gamma / 2, j = 64 kc + 8 g + e
__global__ void k_tt_tile_b(const float* __restrict__ Vt, const int64_t* __restrict__ vt_off,
                            const int4* __restrict__ b_info, const int* __restrict__ Nb,
                            const int64_t* __restrict__ row_off, const float2* __restrict__ f,
                            const float* __restrict__ scale, int64_t n_chunks, __half* __restrict__ B) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_chunks * 8 * 128) return;
  const int gam = int(t % 128), g = int((t / 128) % 8);
  const int64_t chunk = t / (8 * 128);
  const int4 I = b_info[chunk];
  const int N = Nb[I.x], ld = (N + 3) & ~3;
  const int c = I.y * kTtCols + gam / 2;
  const float sb = scale[2 * I.x + 1];
  const float* w = Vt + vt_off[I.x];
  const float2* fb = f + row_off[I.x];
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int j = I.z * 64 + 8 * g + e;
    float v = 0.f;
    if (c < N && j < N) {
      const float2 fj = fb[j];
      v = w[int64_t(j) * ld + c] * ((gam & 1) ? fj.y : fj.x) * sb;
    }
    x[e] = v;
  }
  tt_split8(x, B + tc_b_index(chunk, 0, gam, 8 * g, 128), B + tc_b_index(chunk, 1, gam, 8 * g, 128));
}

static void tt_tables(mtf_system sys, TtForm& t, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  std::vector<int> Ns(m->nd), ldt(m->nd);
  for (int i = 0; i < m->nd; ++i) {
    Ns[i] = m->blk[i].N;
    ldt[i] = m->blk[i].N + (m->blk[i].N & 1);
  }
  const std::string why = plan_tt(Ns, t.plan);
  MTF_REQUIRE(why.empty(), MTF_ERR_MESH, why);
  const TtPlan& p = t.plan;
  std::vector<int4> ai(size_t(p.n_a)), bi(size_t(p.n_b)), un, inf;
  for (int i = 0; i < m->nd; ++i) {
    const TtBlock& q = p.blocks[size_t(i)];
    for (int mt = 0; mt < q.n_mt; ++mt)
      for (int kc = 0; kc < q.n_kc; ++kc) ai[size_t(q.a_base + int64_t(mt) * q.n_kc + kc)] = make_int4(i, mt, kc, 0);
    for (int nt = 0; nt < q.n_nt; ++nt)
      for (int kc = 0; kc < q.n_kc; ++kc) bi[size_t(q.b_base + int64_t(nt) * q.n_kc + kc)] = make_int4(i, nt, kc, 0);
  }
  for (const TtUnit& u : p.units) {
    const TtBlock& q = p.blocks[size_t(u.blk)];
    const int64_t a0 = q.a_base + int64_t(u.mt) * q.n_kc, b0 = q.b_base + int64_t(u.nt) * q.n_kc;
    MTF_REQUIRE(a0 < (int64_t(1) << 31) && b0 < (int64_t(1) << 31), MTF_ERR_MESH, "block-OSRC formation too large");
    un.push_back(make_int4(int(a0), int(b0), 0, q.n_kc));
    inf.push_back(make_int4(u.blk, u.mt * kTcRows, u.nt * kTtCols, 0));
  }
  t.a_info.upload(ai, s);
  t.b_info.upload(bi, s);
  t.units.upload(un, s);
  t.info.upload(inf, s);
  t.N.upload(Ns, s);
  t.ldt.upload(ldt, s);
  t.off.upload(m->os_T_off_h, s);
  std::vector<int64_t> vo(m->osrc_off_h.begin(), m->osrc_off_h.end()), ro(size_t(m->nd));
  for (int i = 0; i < m->nd; ++i) ro[size_t(i)] = m->blk[i].row_off;
  t.vt_off.upload(vo, s);
  t.row_off.upload(ro, s);
  t.scale.alloc(size_t(2 * m->nd));
  t.inv.alloc(size_t(m->nd));
  t.wmax.alloc(size_t(m->n_rows));
  t.A.alloc(size_t(p.n_a) * 2 * kTcRows * 64);
  t.B.alloc(size_t(p.n_b) * 2 * 128 * 64);
  tc_encode_map(&t.amap, t.A.p, kTcRows, 2, p.n_a);
  tc_encode_map(&t.bmap, t.B.p, 128, 2, p.n_b);
  int dev = 0, sms = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  MTF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  t.n_cta = std::max(1, std::min(sms, int(p.units.size())));
  MTF_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
}

// sys->d_osrc_T (interleaved complex rows, stride N_i + (N_i & 1), offsets
// m->os_T_off_h, allocated by the caller) := W_i diag(f_i) W_i^T for every
// block, f = sys->d_osrc_f
void osrc_form_tc(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  if (!sys->tt) sys->tt = new TtForm();
  TtForm& t = *sys->tt;
  if (t.plan.blocks.empty()) tt_tables(sys, t, s);
  const TtPlan& p = t.plan;
  const float2* f = reinterpret_cast<const float2*>(sys->d_osrc_f.p);
  if (!t.a_built) {
    MTF_LAUNCH(KID_TT, s, k_tt_wmax<<<unsigned((m->n_rows * 32 + 255) / 256), 256, 0, s>>>(
        m->d_osrc_Vt.p, t.vt_off.p, m->d_row_blk.p, t.row_off.p, t.N.p, m->n_rows, t.wmax.p));
  }
  MTF_LAUNCH(KID_TT, s, k_tt_scales<<<unsigned(m->nd), 256, 0, s>>>(t.wmax.p, f, t.row_off.p, t.N.p, t.scale.p, t.inv.p));
  if (!t.a_built) {
    const int64_t na = p.n_a * 8 * kTcRows;
    MTF_LAUNCH(KID_TT, s, k_tt_tile_a<<<unsigned((na + 255) / 256), 256, 0, s>>>(
        m->d_osrc_Vt.p, t.vt_off.p, t.a_info.p, t.N.p, t.scale.p, p.n_a, t.A.p));
    t.a_built = true;
  }
  const int64_t nb = p.n_b * 8 * 128;
  MTF_LAUNCH(KID_TT, s, k_tt_tile_b<<<unsigned((nb + 255) / 256), 256, 0, s>>>(
      m->d_osrc_Vt.p, t.vt_off.p, t.b_info.p, t.N.p, t.row_off.p, f, t.scale.p, p.n_b, t.B.p));
  // pads of the rows (N_i odd) stay zero; every other entry is written once
  MTF_CUDA(cudaMemsetAsync(sys->d_osrc_T.p, 0, sys->d_osrc_T.n * sizeof(float), s));
  using Cfg = TcsCfg<2, 128>;
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(opted.load() & bit)) {
    MTF_CUDA(cudaFuncSetAttribute(k_tc_stream<2, 128, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem)));
    opted.fetch_or(bit);
  }
  stream_prepare(sys, s);
  TcUnits units;
  units.list = t.units.p;
  TcTtOut out;
  out.info = t.info.p;
  out.N = t.N.p;
  out.ldt = t.ldt.p;
  out.off = t.off.p;
  out.inv = t.inv.p;
  out.T = reinterpret_cast<float2*>(sys->d_osrc_T.p);
  MTF_LAUNCH(KID_TT_MMA, s, k_tc_stream<2, 128, 2><<<unsigned(t.n_cta), 192, Cfg::smem, s>>>(
      t.amap, t.bmap, units, int(p.units.size()), nullptr, nullptr, nullptr, nullptr, 0, 0, 0, nullptr,
      sys->d_mv_ctl.p + 2, out));
  check_matvec_stream(sys, s);
}

}  // namespace mtf
