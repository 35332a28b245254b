// MTF operator apply y = M x (Problem 2): per block i the dense Calderon
// part 2 A_i u_i = 2 [K u_D + rho^-1 T u_N ; -rho T u_D + K u_N] (Eq. 9)
// fused with the skeleton exchange sum_{j in Lambda_i} G^{ij} u_j applied to
// both trace slots with the same sign (Eqs. 11-13, Remark 2).
//
// One warp per row (block i, dof m): the warp streams row m of the block's
// interleaved (T, K) matrix once per group of four right-hand sides with
// coalesced 32-byte loads, reduces, and its lane 0 adds the six exchange
// entries of the row (two triangles of Gamma_i on edge m, three RWG_j
// functions each).  The kernel is HBM-bound: it moves the matrix once.
#include <algorithm>

#include "common.h"

namespace mtf {

template <class MatT>
struct Entry;
template <>
struct Entry<double> {
  // (T.re, T.im, K.re, K.im) as two 16-byte loads
  static __device__ __forceinline__ void load(const double* row, int n, double& tr, double& ti, double& kr,
                                              double& ki) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(row) + 2 * n);
    const double2 b = __ldg(reinterpret_cast<const double2*>(row) + 2 * n + 1);
    tr = a.x; ti = a.y; kr = b.x; ki = b.y;
  }
};
template <>
struct Entry<float> {
  static __device__ __forceinline__ void load(const float* row, int n, float& tr, float& ti, float& kr,
                                              float& ki) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(row) + n);
    tr = a.x; ti = a.y; kr = a.z; ki = a.w;
  }
};

template <class VecT>
struct VecLoad;
template <>
struct VecLoad<double> {
  static __device__ __forceinline__ double2 ld(const double* p) { return *reinterpret_cast<const double2*>(p); }
};
template <>
struct VecLoad<float> {
  static __device__ __forceinline__ float2 ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
};

// MatT: storage precision of the (T, K) blocks; AccT: arithmetic and
// accumulation precision; VecT: precision of the dense-part input vector xv
// (an FP32 copy of x on the FP32 path, so that no FP64 conversion sits in the
// inner loop).  The exchange part and the output are FP64.
template <class MatT, class AccT, class VecT>
__global__ void __launch_bounds__(256) k_matvec(
    const MatT* __restrict__ TK, const XEntry* __restrict__ xe, const double* __restrict__ xval,
    const int32_t* __restrict__ row_blk, const int64_t* __restrict__ blk_row_off,
    const int32_t* __restrict__ blk_N, const int64_t* __restrict__ blk_dof_off,
    const int64_t* __restrict__ blk_mat_off, const double* __restrict__ rho, const double* __restrict__ x,
    int64_t ldx, const VecT* __restrict__ xv, int64_t ldxv, double* __restrict__ y, int64_t ldy, int nrhs,
    int64_t n_rows) {
  const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  const int i = row_blk[r];
  const int64_t m = r - blk_row_off[i];
  const int N = blk_N[i];
  const int64_t off = blk_dof_off[i];
  const MatT* row = TK + 4 * (blk_mat_off[i] + m * N);
  const double rr = rho[2 * i], ri = rho[2 * i + 1];
  const double rn = rr * rr + ri * ri;
  const double ir = rr / rn, ii = -ri / rn;  // 1 / rho
  for (int c0 = 0; c0 < nrhs; c0 += 4) {
    const int nc = min(4, nrhs - c0);
    AccT acc[4][8];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[c][q] = AccT(0);
    // U row entries per lane in flight: the loads of a group are issued
    // before any of their arithmetic (latency hiding for the HBM stream)
    constexpr int U = sizeof(MatT) == 4 ? 4 : 2;
    for (int n0 = lane; n0 < N; n0 += 32 * U) {
      MatT e[U][4];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int n = n0 + 32 * u;
        if (n < N) Entry<MatT>::load(row, n, e[u][0], e[u][1], e[u][2], e[u][3]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int n = n0 + 32 * u;
        if (n >= N) break;
        const AccT Tr = AccT(e[u][0]), Ti = AccT(e[u][1]), Kr = AccT(e[u][2]), Ki = AccT(e[u][3]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c < nc) {
            const VecT* xc = xv + 2 * (int64_t(c0 + c) * ldxv + off);
            const auto xd2 = VecLoad<VecT>::ld(xc + 2 * n);
            const auto xn2 = VecLoad<VecT>::ld(xc + 2 * (N + n));
            const AccT xdr = AccT(xd2.x), xdi = AccT(xd2.y), xnr = AccT(xn2.x), xni = AccT(xn2.y);
            // T xd, T xn, K xd, K xn
            acc[c][0] += Tr * xdr - Ti * xdi;
            acc[c][1] += Tr * xdi + Ti * xdr;
            acc[c][2] += Tr * xnr - Ti * xni;
            acc[c][3] += Tr * xni + Ti * xnr;
            acc[c][4] += Kr * xdr - Ki * xdi;
            acc[c][5] += Kr * xdi + Ki * xdr;
            acc[c][6] += Kr * xnr - Ki * xni;
            acc[c][7] += Kr * xni + Ki * xnr;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        AccT v = acc[c][q];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
        acc[c][q] = v;
      }
    if (lane < nc) {
      // each of the first nc lanes finishes one right-hand side (in FP64)
      double a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        a[q] = double(acc[0][q]);
#pragma unroll
        for (int c = 1; c < 4; ++c)
          if (lane == c) a[q] = double(acc[c][q]);
      }
      const int col = c0 + lane;
      const double* xc = x + 2 * int64_t(col) * ldx;
      // yD = 2 (Kx + Ty / rho), yN = 2 (-rho Tx + Ky)
      double yDr = 2.0 * (a[4] + (a[2] * ir - a[3] * ii));
      double yDi = 2.0 * (a[5] + (a[2] * ii + a[3] * ir));
      double yNr = 2.0 * (a[6] - (a[0] * rr - a[1] * ri));
      double yNi = 2.0 * (a[7] - (a[0] * ri + a[1] * rr));
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const XEntry X = xe[6 * r + e];
        const double v = xval[6 * r + e];
        const int Nj = X.ab >> 4;
        yDr += v * xc[2 * int64_t(X.col)];
        yDi += v * xc[2 * int64_t(X.col) + 1];
        yNr += v * xc[2 * (int64_t(X.col) + Nj)];
        yNi += v * xc[2 * (int64_t(X.col) + Nj) + 1];
      }
      double* yc = y + 2 * (int64_t(col) * ldy + off);
      yc[2 * m] = yDr;
      yc[2 * m + 1] = yDi;
      yc[2 * (N + m)] = yNr;
      yc[2 * (N + m) + 1] = yNi;
    }
  }
}

// Refinement residual matvec of the mixed path: FP32-stored (T, K), input x
// split into FP32 pairs x = x_hi + x_lo (48 significant bits), and every
// product accumulated in double-float: a x_hi = p + e exactly (e by FMA),
// a x_lo added to e, p added to the running (hi, lo) pair by an error-free
// two-sum.  The sums carry about 2^-46 relative error against a few times
// 2^-53 for FP64 FMAs, at FP32 throughput instead of the narrow FP64 pipe.
// Lanes convert to FP64 for the warp reduction and the FP64 epilogue (rho,
// exchange), as k_matvec does.
// (the _rn intrinsics keep the compiler from contracting the product into
// the sum, which would break the error-free transformations)
__device__ __forceinline__ void df_mac(float& hi, float& lo, float a, float xh, float xl) {
  const float p = __fmul_rn(a, xh);
  float e = fmaf(a, xh, -p);  // exact: a xh = p + e
  e = fmaf(a, xl, e);
  const float s = __fadd_rn(hi, p);  // two-sum of hi and p
  const float z = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// E64: the operator is the FP64 blocks, given as FP32 pairs (TK = fl(v),
// TKlo = fl(v - fl(v)), split once per assembly): every product adds the
// lo part times the input's hi part to the running lo sum, so the residual
// of the FP64-assembled system costs FP32 work (residual_fp64).
template <bool E64>
__global__ void __launch_bounds__(256) k_matvec_df(
    const float* __restrict__ TK, const float* __restrict__ TKlo, const XEntry* __restrict__ xe,
    const double* __restrict__ xval,
    const int32_t* __restrict__ row_blk, const int64_t* __restrict__ blk_row_off,
    const int32_t* __restrict__ blk_N, const int64_t* __restrict__ blk_dof_off,
    const int64_t* __restrict__ blk_mat_off, const double* __restrict__ rho, const double* __restrict__ x,
    int64_t ldx, const float* __restrict__ xh, const float* __restrict__ xl, int64_t ldxv, double* __restrict__ y,
    int64_t ldy, int nrhs, int64_t n_rows) {
  const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  const int i = row_blk[r];
  const int64_t m = r - blk_row_off[i];
  const int N = blk_N[i];
  const int64_t off = blk_dof_off[i];
  const float* row = TK + 4 * (blk_mat_off[i] + m * N);
  const float* rowlo = E64 ? TKlo + 4 * (blk_mat_off[i] + m * N) : nullptr;
  const double rr = rho[2 * i], ri = rho[2 * i + 1];
  const double rn = rr * rr + ri * ri;
  const double ir = rr / rn, ii = -ri / rn;  // 1 / rho
  for (int c0 = 0; c0 < nrhs; c0 += 2) {
    const int nc = min(2, nrhs - c0);
    float ah[2][8], al[2][8];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q) ah[c][q] = al[c][q] = 0.f;
    constexpr int U = 4;
    for (int n0 = lane; n0 < N; n0 += 32 * U) {
      float4 e[U], el[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int n = n0 + 32 * u;
        if (n < N) {
          e[u] = __ldg(reinterpret_cast<const float4*>(row) + n);
          if constexpr (E64) el[u] = __ldg(reinterpret_cast<const float4*>(rowlo) + n);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int n = n0 + 32 * u;
        if (n >= N) break;
        const float Tr = e[u].x, Ti = e[u].y, Kr = e[u].z, Ki = e[u].w;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (c < nc) {
            const int64_t o = 2 * (int64_t(c0 + c) * ldxv + off);
            const float2 dh = *reinterpret_cast<const float2*>(xh + o + 2 * n);
            const float2 dl = *reinterpret_cast<const float2*>(xl + o + 2 * n);
            const float2 nh = *reinterpret_cast<const float2*>(xh + o + 2 * (N + n));
            const float2 nl = *reinterpret_cast<const float2*>(xl + o + 2 * (N + n));
            float* H = ah[c];
            float* Lo = al[c];
            // T xd, T xn, K xd, K xn
            df_mac(H[0], Lo[0], Tr, dh.x, dl.x);
            df_mac(H[0], Lo[0], -Ti, dh.y, dl.y);
            df_mac(H[1], Lo[1], Tr, dh.y, dl.y);
            df_mac(H[1], Lo[1], Ti, dh.x, dl.x);
            df_mac(H[2], Lo[2], Tr, nh.x, nl.x);
            df_mac(H[2], Lo[2], -Ti, nh.y, nl.y);
            df_mac(H[3], Lo[3], Tr, nh.y, nl.y);
            df_mac(H[3], Lo[3], Ti, nh.x, nl.x);
            df_mac(H[4], Lo[4], Kr, dh.x, dl.x);
            df_mac(H[4], Lo[4], -Ki, dh.y, dl.y);
            df_mac(H[5], Lo[5], Kr, dh.y, dl.y);
            df_mac(H[5], Lo[5], Ki, dh.x, dl.x);
            df_mac(H[6], Lo[6], Kr, nh.x, nl.x);
            df_mac(H[6], Lo[6], -Ki, nh.y, nl.y);
            df_mac(H[7], Lo[7], Kr, nh.y, nl.y);
            df_mac(H[7], Lo[7], Ki, nh.x, nl.x);
            if constexpr (E64) {
              // the entries' lo parts times the inputs' hi parts
              const float tr = el[u].x, ti = el[u].y, kr = el[u].z, ki = el[u].w;
              Lo[0] = fmaf(tr, dh.x, fmaf(-ti, dh.y, Lo[0]));
              Lo[1] = fmaf(tr, dh.y, fmaf(ti, dh.x, Lo[1]));
              Lo[2] = fmaf(tr, nh.x, fmaf(-ti, nh.y, Lo[2]));
              Lo[3] = fmaf(tr, nh.y, fmaf(ti, nh.x, Lo[3]));
              Lo[4] = fmaf(kr, dh.x, fmaf(-ki, dh.y, Lo[4]));
              Lo[5] = fmaf(kr, dh.y, fmaf(ki, dh.x, Lo[5]));
              Lo[6] = fmaf(kr, nh.x, fmaf(-ki, nh.y, Lo[6]));
              Lo[7] = fmaf(kr, nh.y, fmaf(ki, nh.x, Lo[7]));
            }
          }
        }
      }
    }
    double acc[2][8];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        double v = double(ah[c][q]) + double(al[c][q]);
#pragma unroll
        for (int s2 = 16; s2 > 0; s2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s2);
        acc[c][q] = v;
      }
    if (lane < nc) {
      double a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = lane == 0 ? acc[0][q] : acc[1][q];
      const int col = c0 + lane;
      const double* xc = x + 2 * int64_t(col) * ldx;
      // yD = 2 (Kx + Ty / rho), yN = 2 (-rho Tx + Ky)
      double yDr = 2.0 * (a[4] + (a[2] * ir - a[3] * ii));
      double yDi = 2.0 * (a[5] + (a[2] * ii + a[3] * ir));
      double yNr = 2.0 * (a[6] - (a[0] * rr - a[1] * ri));
      double yNi = 2.0 * (a[7] - (a[0] * ri + a[1] * rr));
#pragma unroll
      for (int e2 = 0; e2 < 6; ++e2) {
        const XEntry X = xe[6 * r + e2];
        const double v = xval[6 * r + e2];
        const int Nj = X.ab >> 4;
        yDr += v * xc[2 * int64_t(X.col)];
        yDi += v * xc[2 * int64_t(X.col) + 1];
        yNr += v * xc[2 * (int64_t(X.col) + Nj)];
        yNi += v * xc[2 * (int64_t(X.col) + Nj) + 1];
      }
      double* yc = y + 2 * (int64_t(col) * ldy + off);
      yc[2 * m] = yDr;
      yc[2 * m + 1] = yDi;
      yc[2 * (N + m)] = yNr;
      yc[2 * (N + m) + 1] = yNi;
    }
  }
}

// x (FP64, column stride ldx) -> FP32 pair hi = fl(x), lo = fl(x - hi), n2
// reals per column, columns packed
__global__ void k_split_f32(const double* __restrict__ x, int64_t ldx, int64_t n2, int nrhs, float* __restrict__ hi,
                            float* __restrict__ lo) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n2 * nrhs) return;
  const int64_t c = t / n2, k = t % n2;
  const double v = x[2 * c * ldx + k];
  const float h = float(v);
  hi[t] = h;
  lo[t] = float(v - double(h));
}

__global__ void k_to_f32(const double* __restrict__ x, int64_t ldx, int64_t n2, int nrhs, float* __restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n2 * nrhs) return;
  const int64_t c = t / n2, k = t % n2;
  out[t] = float(x[2 * c * ldx + k]);
}

void launch_matvec_kind(mtf_system sys, int kind, const double* x, int64_t ldx, double* y, int64_t ldy,
                        int nrhs, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const unsigned blocks = unsigned((m->n_rows * 32 + 255) / 256);
  if (kind == MV_AUTO) kind = sys->opt.precision == MTF_PREC_FP64 ? MV_FP64 : MV_FP32;
  if (kind == MV_FP64 && sys->opt.precision != MTF_PREC_FP64 && sys->d_TK64hl.p) {
    // mixed path with residual_fp64: the FP64 blocks as FP32 pairs, double-float sums
    const int64_t n2 = 2 * m->n_total;
    if (sys->d_x32.n < 2 * size_t(n2) * nrhs) sys->d_x32.alloc(2 * size_t(n2) * nrhs);
    float* xh = sys->d_x32.p;
    float* xl = xh + size_t(n2) * nrhs;
    MTF_LAUNCH(KID_MISC, s, k_split_f32<<<unsigned((n2 * nrhs + 255) / 256), 256, 0, s>>>(x, ldx, n2, nrhs, xh, xl));
    MTF_LAUNCH(KID_MATVEC64, s, k_matvec_df<true><<<blocks, 256, 0, s>>>(
        sys->d_TK64hl.p, sys->d_TK64hl.p + size_t(m->n_mat) * 4, m->d_xent.p, sys->d_xval.p, m->d_row_blk.p,
        m->d_blk_row_off.p, m->d_blk_N.p, m->d_blk_dof_off.p, m->d_blk_mat_off.p, sys->d_rho.p, x, ldx, xh, xl,
        m->n_total, y, ldy, nrhs, m->n_rows));
  } else if (kind == MV_FP64) {
    MTF_LAUNCH(KID_MATVEC64, s, k_matvec<double, double, double><<<blocks, 256, 0, s>>>(
        sys->d_TK64.p, m->d_xent.p, sys->d_xval.p, m->d_row_blk.p, m->d_blk_row_off.p, m->d_blk_N.p,
        m->d_blk_dof_off.p, m->d_blk_mat_off.p, sys->d_rho.p, x, ldx, x, ldx, y, ldy, nrhs, m->n_rows));
  } else if (kind == MV_FP32) {
    const int64_t n2 = 2 * m->n_total;
    if (sys->d_x32.n < size_t(n2) * nrhs) sys->d_x32.alloc(size_t(n2) * nrhs);
    MTF_LAUNCH(KID_MISC, s, k_to_f32<<<unsigned((n2 * nrhs + 255) / 256), 256, 0, s>>>(x, ldx, n2, nrhs, sys->d_x32.p));
    launch_matvec_stream64(sys, x, ldx, sys->d_x32.p, m->n_total, y, ldy, nrhs, s);
  } else if (sys->opt.residual_df) {
    // FP32 storage, double-float sums of the split input
    const int64_t n2 = 2 * m->n_total;
    if (sys->d_x32.n < 2 * size_t(n2) * nrhs) sys->d_x32.alloc(2 * size_t(n2) * nrhs);
    float* xh = sys->d_x32.p;
    float* xl = xh + size_t(n2) * nrhs;
    MTF_LAUNCH(KID_MISC, s, k_split_f32<<<unsigned((n2 * nrhs + 255) / 256), 256, 0, s>>>(x, ldx, n2, nrhs, xh, xl));
    MTF_LAUNCH(KID_MATVEC64, s, k_matvec_df<false><<<blocks, 256, 0, s>>>(
        sys->d_TK32.p, nullptr, m->d_xent.p, sys->d_xval.p, m->d_row_blk.p, m->d_blk_row_off.p, m->d_blk_N.p,
        m->d_blk_dof_off.p, m->d_blk_mat_off.p, sys->d_rho.p, x, ldx, xh, xl, m->n_total, y, ldy, nrhs, m->n_rows));
  } else {
    MTF_LAUNCH(KID_MATVEC64, s, k_matvec<float, double, double><<<blocks, 256, 0, s>>>(
        sys->d_TK32.p, m->d_xent.p, sys->d_xval.p, m->d_row_blk.p, m->d_blk_row_off.p, m->d_blk_N.p,
        m->d_blk_dof_off.p, m->d_blk_mat_off.p, sys->d_rho.p, x, ldx, x, ldx, y, ldy, nrhs, m->n_rows));
  }
}

// y = M x with the operator as stored: FP64 storage and arithmetic on the FP64
// path and on the mixed path with residual_fp64; FP32 storage with
// double-float accumulation of the FP64 input (the refinement residual) on
// the mixed path otherwise.
void launch_matvec(mtf_system sys, const double* x, int64_t ldx, double* y, int64_t ldy, int nrhs,
                   cudaStream_t s) {
  const bool fp64 = sys->opt.precision == MTF_PREC_FP64 || sys->opt.residual_fp64;
  launch_matvec_kind(sys, fp64 ? MV_FP64 : MV_FP32_ACC64, x, ldx, y, ldy, nrhs, s);
}

}  // namespace mtf
