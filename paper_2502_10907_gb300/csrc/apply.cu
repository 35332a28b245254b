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
#include "common.h"

namespace mtf {

struct C2m {
  double re, im;
};

__global__ void __launch_bounds__(256) k_matvec64(
    const double* __restrict__ TK, const XEntry* __restrict__ xe, const double* __restrict__ xval,
    const int32_t* __restrict__ row_blk, const int64_t* __restrict__ blk_row_off,
    const int32_t* __restrict__ blk_N, const int64_t* __restrict__ blk_dof_off,
    const int64_t* __restrict__ blk_mat_off, const double* __restrict__ rho, const double* __restrict__ x,
    int64_t ldx, double* __restrict__ y, int64_t ldy, int nrhs, int64_t n_rows) {
  const int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  const int i = row_blk[r];
  const int64_t m = r - blk_row_off[i];
  const int N = blk_N[i];
  const int64_t off = blk_dof_off[i];
  const double2* row = reinterpret_cast<const double2*>(TK + 4 * (blk_mat_off[i] + m * N));
  const double rr = rho[2 * i], ri = rho[2 * i + 1];
  const double rn = rr * rr + ri * ri;
  const double ir = rr / rn, ii = -ri / rn;  // 1 / rho
  for (int c0 = 0; c0 < nrhs; c0 += 4) {
    const int nc = min(4, nrhs - c0);
    double acc[4][8];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[c][q] = 0.0;
    for (int n = lane; n < N; n += 32) {
      const double2 t2 = __ldg(row + 2 * n), k2 = __ldg(row + 2 * n + 1);
      const double4 tk = make_double4(t2.x, t2.y, k2.x, k2.y);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < nc) {
          const double* xc = x + 2 * (int64_t(c0 + c) * ldx + off);
          const double2 xd = *reinterpret_cast<const double2*>(xc + 2 * n);
          const double2 xn = *reinterpret_cast<const double2*>(xc + 2 * (N + n));
          // T xd, T xn, K xd, K xn
          acc[c][0] += tk.x * xd.x - tk.y * xd.y;
          acc[c][1] += tk.x * xd.y + tk.y * xd.x;
          acc[c][2] += tk.x * xn.x - tk.y * xn.y;
          acc[c][3] += tk.x * xn.y + tk.y * xn.x;
          acc[c][4] += tk.z * xd.x - tk.w * xd.y;
          acc[c][5] += tk.z * xd.y + tk.w * xd.x;
          acc[c][6] += tk.z * xn.x - tk.w * xn.y;
          acc[c][7] += tk.z * xn.y + tk.w * xn.x;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        double v = acc[c][q];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
        acc[c][q] = v;
      }
    if (lane < nc) {
      // each of the first nc lanes finishes one right-hand side
      double a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        a[q] = acc[0][q];
#pragma unroll
        for (int c = 1; c < 4; ++c)
          if (lane == c) a[q] = acc[c][q];
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

void launch_matvec(mtf_system sys, const double* x, int64_t ldx, double* y, int64_t ldy, int nrhs,
                   cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const int64_t threads = m->n_rows * 32;
  MTF_LAUNCH(KID_MATVEC64, s, k_matvec64<<<unsigned((threads + 255) / 256), 256, 0, s>>>(
      sys->d_TK64.p, m->d_xent.p, sys->d_xval.p, m->d_row_blk.p, m->d_blk_row_off.p, m->d_blk_N.p,
      m->d_blk_dof_off.p, m->d_blk_mat_off.p, sys->d_rho.p, x, ldx, y, ldy, nrhs, m->n_rows));
  MTF_CUDA(cudaGetLastError());
}

}  // namespace mtf
