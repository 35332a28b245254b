// FP32 block matvec of the mixed inner solver (Eq. 16 applied as
// y = 2 A x + X x, block by block, as in the FP64 kernel): the stored
// {T, K} entries are streamed by the bulk-copy row kernel of stream.cuh
// (ENT = 2); k_mv_combine adds each row's pieces and applies the epilogue.
#include <algorithm>

#include "stream.cuh"

namespace mtf {

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
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  constexpr int K = StreamK<NC, 2>::K;
  using AT = YT;
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int i = row_blk[row];
  const int N = blk_N[i];
  const int P = st_pieces<2>(N);
  const float tot = st_row_total<K>(part + row * pmax * K, P, lane);
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

// Adjoint epilogue (FP32): the streamed partial sums were taken against
// a = conj(v_D), b = conj(v_N); with T and K complex symmetric (Galerkin
// forms of symmetric kernels, assembled symmetric to rounding) and the
// exchange matrix X real symmetric,
//   (M^H v)_D = conj(2 (K a - rho T b)) + X v_D-slots,
//   (M^H v)_N = conj(2 (T a / rho + K b)) + X v_N-slots.
template <int NC>
__global__ void __launch_bounds__(256) k_mv_combine_adj(
    const float* __restrict__ part, int pmax, const int32_t* __restrict__ row_blk, const int32_t* __restrict__ blk_N,
    const int64_t* __restrict__ blk_dof_off, const int64_t* __restrict__ blk_row_off, const XEntry* __restrict__ xe,
    const float* __restrict__ xval32, const float* __restrict__ rho32, const float* __restrict__ v, int64_t ldv,
    float* __restrict__ y, int64_t ldy, int c0, int64_t n_rows) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  constexpr int K = StreamK<NC, 2>::K;
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int i = row_blk[row];
  const int N = blk_N[i];
  const float tot = st_row_total<K>(part + row * pmax * K, st_pieces<2>(N), lane);
  float a[8];
  const int cl = lane < NC ? lane : 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = __shfl_sync(0xffffffffu, tot, cl * 8 + q);
  if (lane >= NC) return;
  const int64_t m = row - blk_row_off[i];
  const int64_t off = blk_dof_off[i];
  const float rr = rho32[4 * i], ri = rho32[4 * i + 1], ir = rho32[4 * i + 2], ii = rho32[4 * i + 3];
  const int col = c0 + lane;
  const float* vc = v + 2 * int64_t(col) * ldv;
  // P_D = K a - rho T b, P_N = T a / rho + K b
  const float pDr = a[4] - (rr * a[2] - ri * a[3]), pDi = a[5] - (rr * a[3] + ri * a[2]);
  const float pNr = ir * a[0] - ii * a[1] + a[6], pNi = ir * a[1] + ii * a[0] + a[7];
  float yDr = 2.f * pDr, yDi = -2.f * pDi, yNr = 2.f * pNr, yNi = -2.f * pNi;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const XEntry X = xe[6 * row + e];
    const float xv = xval32[6 * row + e];
    const int Nj = X.ab >> 4;
    yDr += xv * vc[2 * int64_t(X.col)];
    yDi += xv * vc[2 * int64_t(X.col) + 1];
    yNr += xv * vc[2 * (int64_t(X.col) + Nj)];
    yNi += xv * vc[2 * (int64_t(X.col) + Nj) + 1];
  }
  float* yc = y + 2 * (int64_t(col) * ldy + off);
  yc[2 * m] = yDr;
  yc[2 * m + 1] = yDi;
  yc[2 * (N + m)] = yNr;
  yc[2 * (N + m) + 1] = yNi;
}

// out^c = conj(v^c) over n complex entries (column strides ldv, ldo)
__global__ void k_conj32(const float* __restrict__ v, int64_t ldv, int64_t n, float* __restrict__ out, int64_t ldo) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 x = reinterpret_cast<const float2*>(v + 2 * int64_t(c) * ldv)[k];
  reinterpret_cast<float2*>(out + 2 * int64_t(c) * ldo)[k] = make_float2(x.x, -x.y);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
void build_stream_units(mtf_mesh m, int rows, int piece_len, int entry_bytes, const std::vector<int64_t>& blk_entry_off,
                        const std::vector<int64_t>& row_stride, StreamUnits& su, cudaStream_t s) {
  std::vector<StreamBlock> blocks(static_cast<size_t>(m->nd));
  for (int i = 0; i < m->nd; ++i) {
    blocks[size_t(i)].N = m->blk[i].N;
    blocks[size_t(i)].row_off = m->blk[i].row_off;
    blocks[size_t(i)].dof_off = m->blk[i].dof_off;
    blocks[size_t(i)].entry_off = blk_entry_off[i];
    blocks[size_t(i)].ld = row_stride[i];
  }
  StreamPlan plan;
  const std::string why = plan_stream_units(blocks, rows, piece_len, entry_bytes, plan);
  MTF_REQUIRE(why.empty(), MTF_ERR_MESH, why);
  MTF_REQUIRE(m->n_total < (int64_t(1) << 31), MTF_ERR_MESH, "mesh too large for the streaming tables");
  const size_t nu = size_t(plan.n_units());
  su.n_units = plan.n_units();
  su.pmax = plan.pmax;
  su.tiled_bytes = plan.tiled_bytes;
  su.d_units.alloc(nu);
  su.d_src.alloc(nu);
  su.d_toff.alloc(nu);
  if (nu > 0) {
    static_assert(sizeof(int4) == 4 * sizeof(int32_t), "unit records are four int32");
    MTF_CUDA(cudaMemcpyAsync(su.d_units.p, plan.rec.data(), nu * sizeof(int4), cudaMemcpyHostToDevice, s));
    MTF_CUDA(cudaMemcpyAsync(su.d_src.p, plan.src.data(), nu * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MTF_CUDA(cudaMemcpyAsync(su.d_toff.p, plan.toff.data(), nu * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MTF_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  }
  su.ready = true;
}

// Tiled copy of a streamed operator: unit u's nrows rows at byte offset
// toff[u] with the pitch st_tile_pitch(eb, len), each row the unit's entries
// (whole 16-byte words of the dense row, which stay inside it: the units
// table checks that) followed by zeros up to the pitch.  One CTA per unit.
__global__ void k_tile_units(const unsigned char* __restrict__ dense, const int4* __restrict__ units,
                             const int64_t* __restrict__ usrc, const int64_t* __restrict__ toff, int eb,
                             unsigned char* __restrict__ tiled) {
  const int u = blockIdx.x;
  const int4 rec = units[u];
  const int N = rec.x, len = rec.w & 0xfff, nrows = (rec.w >> 24) & 0xff;
  const int pitch = st_tile_pitch(eb, len), words = pitch / 16, used = len * eb;
  const int64_t ld = eb == 16 ? N : (eb == 8 ? N + (N & 1) : (N + 3) & ~3);
  const int64_t src = usrc[u] * eb, dst = toff[u];
  for (int t = threadIdx.x; t < nrows * words; t += blockDim.x) {
    const int r = t / words, w = t - r * words;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (w * 16 < used) v = *reinterpret_cast<const uint4*>(dense + src + int64_t(r) * ld * eb + w * 16);
    *reinterpret_cast<uint4*>(tiled + dst + int64_t(r) * pitch + w * 16) = v;
  }
}

void tile_stream_operator(const StreamUnits& su, const void* dense, int eb, void* tiled, cudaStream_t s) {
  MTF_REQUIRE(su.ready && (reinterpret_cast<uintptr_t>(dense) & 15) == 0 && (reinterpret_cast<uintptr_t>(tiled) & 15) == 0,
              MTF_ERR_ARG, "tiled operator copy needs built units and 16-byte aligned buffers");
  if (su.n_units == 0) return;
  MTF_LAUNCH(KID_MISC, s, k_tile_units<<<unsigned(su.n_units), 256, 0, s>>>(
      static_cast<const unsigned char*>(dense), su.d_units.p, su.d_src.p, su.d_toff.p, eb,
      static_cast<unsigned char*>(tiled)));
}

void stream_prepare(mtf_system sys, cudaStream_t s) {
  if (!sys->d_mv_ctl.p) {
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

static void ensure_mv_scratch(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  stream_prepare(sys, s);
  if (!m->mv_units.ready) {
    std::vector<int64_t> off(m->nd), ld(m->nd);
    for (int i = 0; i < m->nd; ++i) {
      off[i] = m->blk[i].mat_off;
      ld[i] = m->blk[i].N;
    }
    build_stream_units(m, st_unit_rows<2>(), st_piece_len<2>(), 16, off, ld, m->mv_units, s);
  }
  const size_t npart = size_t(m->n_rows) * m->mv_units.pmax * 32;
  if (sys->d_mv_part.n < npart) sys->d_mv_part.alloc(npart);
}

// tiled copy of the FP32 {T, K} entries for the streaming matvec, rebuilt
// after every mixed-precision assembly (MTF_MV_TILED = 0 streams the dense rows)
#ifndef MTF_MV_TILED
#define MTF_MV_TILED 1
#endif
void tile_matvec_operator(mtf_system sys, cudaStream_t s) {
  if (!MTF_MV_TILED) return;
  ensure_mv_scratch(sys, s);
  const StreamUnits& su = sys->mesh->mv_units;
  sys->d_TK32t.alloc(size_t(su.tiled_bytes / 4));
  tile_stream_operator(su, sys->d_TK32.p, 16, sys->d_TK32t.p, s);
}

template <int NC, class XT, class YT>
static void mv_launch(mtf_system sys, const XT* x, int64_t ldx, const float* x32, int64_t ld32, YT* y, int64_t ldy,
                      int c0, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const bool tiled = sys->d_TK32t.p != nullptr;
  launch_stream_tiles<NC, 2>(sys, tiled ? static_cast<const float*>(sys->d_TK32t.p) : sys->d_TK32.p, m->mv_units, x32, ld32, c0,
                             sys->d_mv_part.p, KID_MATVEC32, s, tiled);
  MTF_LAUNCH(KID_MVCOMBINE, s,
             launch_pdl(k_mv_combine<NC, XT, YT>, dim3(unsigned((m->n_rows * 32 + 255) / 256)), dim3(256), 0, s,
                        sys->d_mv_part.p, m->mv_units.pmax, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p,
                        m->d_blk_row_off.p, m->d_xent.p, sys->d_xval.p, sys->d_xval32.p, sys->d_rho.p,
                        sys->d_rho32.p, x, ldx, y, ldy, c0, m->n_rows));
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
  // one FMA pass (up to 4 right-hand sides) beats the tensor-core pass,
  // whose input packing and combine cost more at that width
  if (tc_wide_apply(sys, nrhs)) {
    launch_matvec_tc(sys, x, ldx, y, ldy, nrhs, s);
    return;
  }
  mv_all<float, float>(sys, x, ldx, x, ldx, y, ldy, nrhs, s);
}

template <int NC>
static void mv_adj_launch(mtf_system sys, const float* v, int64_t ldv, const float* a32, int64_t lda, float* y,
                          int64_t ldy, int c0, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const bool tiled = sys->d_TK32t.p != nullptr;
  launch_stream_tiles<NC, 2>(sys, tiled ? static_cast<const float*>(sys->d_TK32t.p) : sys->d_TK32.p, m->mv_units, a32, lda, c0,
                             sys->d_mv_part.p, KID_MATVEC32, s, tiled);
  MTF_LAUNCH(KID_MVCOMBINE, s, k_mv_combine_adj<NC><<<unsigned((m->n_rows * 32 + 255) / 256), 256, 0, s>>>(
      sys->d_mv_part.p, m->mv_units.pmax, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p, m->d_blk_row_off.p,
      m->d_xent.p, sys->d_xval32.p, sys->d_rho32.p, v, ldv, y, ldy, c0, m->n_rows));
}

void launch_conj32(const float* v, int64_t ldv, int64_t n, int ncols, float* out, int64_t ldo, cudaStream_t s) {
  MTF_LAUNCH(KID_MISC, s, k_conj32<<<dim3(unsigned((n + 255) / 256), unsigned(ncols)), 256, 0, s>>>(v, ldv, n, out, ldo));
}

void launch_matvec_adj_f32(mtf_system sys, const float* v, int64_t ldv, float* y, int64_t ldy, int nrhs,
                           cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  ensure_mv_scratch(sys, s);
  const int64_t n = m->n_total;
  if (sys->d_adj32.n < size_t(2 * n) * nrhs) sys->d_adj32.alloc(size_t(2 * n) * nrhs);
  MTF_LAUNCH(KID_MISC, s, k_conj32<<<dim3(unsigned((n + 255) / 256), unsigned(nrhs)), 256, 0, s>>>(
      v, ldv, n, sys->d_adj32.p, n));
  for (int c0 = 0; c0 < nrhs; c0 += 4) {
    const int nc = std::min(4, nrhs - c0);
    if (nc == 1) mv_adj_launch<1>(sys, v, ldv, sys->d_adj32.p, n, y, ldy, c0, s);
    else if (nc == 2) mv_adj_launch<2>(sys, v, ldv, sys->d_adj32.p, n, y, ldy, c0, s);
    else if (nc == 3) mv_adj_launch<3>(sys, v, ldv, sys->d_adj32.p, n, y, ldy, c0, s);
    else mv_adj_launch<4>(sys, v, ldv, sys->d_adj32.p, n, y, ldy, c0, s);
  }
}

// Throws MTF_ERR_TIMEOUT if a launch of a streaming kernel (matvec or OSRC
// apply) gave up on a bulk copy since the last check (synchronises the
// stream) and clears the error word.
void check_matvec_stream(mtf_system sys, cudaStream_t s) {
  if (!sys->d_mv_ctl.p) return;
  unsigned ctl[4];
  MTF_CUDA(cudaMemcpyAsync(ctl, sys->d_mv_ctl.p, sizeof(ctl), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  if (ctl[2] == 0) return;
  MTF_CUDA(cudaMemsetAsync(sys->d_mv_ctl.p, 0, 4 * sizeof(unsigned), s));
  MTF_CUDA(cudaStreamSynchronize(s));
  throw Error{MTF_ERR_TIMEOUT, "a bulk copy of a streaming operator apply did not complete in time"};
}

}  // namespace mtf
