// Galerkin assembly kernels of the MTF operator (Sec. 2.3, Sec. 3.2).
//
// Per block i the library builds the dense EFIO T_i and MFIO K_i Galerkin
// matrices at k_i, tested with the x-pairing (Eq. 5):
//   T[m,n] = -i k int int G psi_n(y).psi_m(x) - 1/(i k) int int G div psi_n div psi_m
//   K[m,n] = -int int grad_x G(x,y) . (psi_n(y) x psi_m(x))
// (Eq. 7 potentials, Eq. 9 operators; the normal cancels in the pairing).
// Entries are stored row-major per block as (T.re, T.im, K.re, K.im).
//
// Each triangle pair (tau test, sigma trial) contributes a 3x3 block.  The
// kernels never form the 9 products per quadrature point: with local origins
// o_tau, o_sigma, x' = x - o_tau, y' = y - o_sigma, Delta = o_tau - o_sigma,
// and RWG functions c_a (x - p_a), c_b (y - q_b), all 18 entries follow from
// 16 complex moments of the kernel over the pair's points,
//   S0 = sum W G, Sx = sum W G x', Sy = sum W G y', Sxy = sum W G x'.y',
//   Q = sum W g, Gx = sum W g x', Gy = sum W g y', C = sum W g (x' x y'),
// g = G (i k - 1/r) / r, through
//   T_ab = c_a c_b [ -ik (Sxy - q'.Sx - p'.Sy + (p'.q') S0) - 4/(ik) S0 ]
//   K_ab = -c_a c_b [ (q' - p' - Delta).C - p'.(Delta x Gy) - q'.(Gx x Delta)
//                     + (q' x p').(Gx - Gy + Delta Q) ]
// (expansion of (x - y).((y - q_b) x (x - p_a)) by the triple product).
#include <cmath>

#include "common.h"

namespace mtf {

__constant__ double c_tri_s[6], c_tri_t[6], c_tri_w[6];  // 6-point rule

#define INV_FOUR_PI 0.079577471545947667884

struct C2 {
  double re, im;
};
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C2 cscale(C2 a, double s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return {a.re - b.re, a.im - b.im}; }

struct Moments {
  C2 S0, Sx[3], Sy[3], Sxy, Q, Gx[3], Gy[3], C[3];
};

__device__ __forceinline__ void zero(Moments& M) {
  C2 z{0, 0};
  M.S0 = M.Sxy = M.Q = z;
  for (int c = 0; c < 3; ++c) M.Sx[c] = M.Sy[c] = M.Gx[c] = M.Gy[c] = M.C[c] = z;
}

// G = exp(i k r) / (4 pi r) and g = G (i k - 1/r) / r for complex k.
__device__ __forceinline__ void helmholtz(double kr, double ki, double r, C2& G, C2& g) {
  const double rinv = 1.0 / r;
  double sn, cs;
  sincos(kr * r, &sn, &cs);
  double amp = INV_FOUR_PI * rinv;
  if (ki != 0.0) amp *= exp(-ki * r);
  G = {amp * cs, amp * sn};
  const C2 f{-ki - rinv, kr};  // i k - 1/r
  g = cscale(cmul(G, f), rinv);
}

// 3x3 local T and K of one pair from its moments; (a, b) = (row, col).
__device__ __forceinline__ void local_entry(const Moments& M, const double* pa, const double* qb,
                                            const double* D, double cc, double kr, double ki, C2& T,
                                            C2& K) {
  const double pq = pa[0] * qb[0] + pa[1] * qb[1] + pa[2] * qb[2];
  C2 X = M.Sxy;
  for (int c = 0; c < 3; ++c) {
    X = csub(X, cscale(M.Sx[c], qb[c]));
    X = csub(X, cscale(M.Sy[c], pa[c]));
  }
  X = cadd(X, cscale(M.S0, pq));
  // -i k X  and  -4/(i k) S0 = 4 i conj(k) / |k|^2 S0
  const C2 mik{ki, -kr};
  const double k2 = kr * kr + ki * ki;
  const C2 f4{4.0 * ki / k2, 4.0 * kr / k2};
  T = cscale(cadd(cmul(mik, X), cmul(f4, M.S0)), cc);
  // K
  double u[3], qxp[3], DxGy_re[3], DxGy_im[3], GxxD_re[3], GxxD_im[3];
  for (int c = 0; c < 3; ++c) u[c] = qb[c] - pa[c] - D[c];
  qxp[0] = qb[1] * pa[2] - qb[2] * pa[1];
  qxp[1] = qb[2] * pa[0] - qb[0] * pa[2];
  qxp[2] = qb[0] * pa[1] - qb[1] * pa[0];
  // Delta x Gy and Gx x Delta
  DxGy_re[0] = D[1] * M.Gy[2].re - D[2] * M.Gy[1].re;
  DxGy_re[1] = D[2] * M.Gy[0].re - D[0] * M.Gy[2].re;
  DxGy_re[2] = D[0] * M.Gy[1].re - D[1] * M.Gy[0].re;
  DxGy_im[0] = D[1] * M.Gy[2].im - D[2] * M.Gy[1].im;
  DxGy_im[1] = D[2] * M.Gy[0].im - D[0] * M.Gy[2].im;
  DxGy_im[2] = D[0] * M.Gy[1].im - D[1] * M.Gy[0].im;
  GxxD_re[0] = M.Gx[1].re * D[2] - M.Gx[2].re * D[1];
  GxxD_re[1] = M.Gx[2].re * D[0] - M.Gx[0].re * D[2];
  GxxD_re[2] = M.Gx[0].re * D[1] - M.Gx[1].re * D[0];
  GxxD_im[0] = M.Gx[1].im * D[2] - M.Gx[2].im * D[1];
  GxxD_im[1] = M.Gx[2].im * D[0] - M.Gx[0].im * D[2];
  GxxD_im[2] = M.Gx[0].im * D[1] - M.Gx[1].im * D[0];
  C2 s{0, 0};
  for (int c = 0; c < 3; ++c) {
    s = cadd(s, cscale(M.C[c], u[c]));
    s.re -= pa[c] * DxGy_re[c] + qb[c] * GxxD_re[c];
    s.im -= pa[c] * DxGy_im[c] + qb[c] * GxxD_im[c];
    const C2 Dm = cadd(csub(M.Gx[c], M.Gy[c]), cscale(M.Q, D[c]));
    s = cadd(s, cscale(Dm, qxp[c]));
  }
  K = cscale(s, -cc);
}

__device__ __forceinline__ void add_entry(double* TK, int64_t idx, C2 T, C2 K) {
  double* e = TK + 4 * idx;
  atomicAdd(e + 0, T.re);
  atomicAdd(e + 1, T.im);
  atomicAdd(e + 2, K.re);
  atomicAdd(e + 3, K.im);
}
__device__ __forceinline__ void add_entry(float* TK, int64_t idx, C2 T, C2 K) {
  atomicAdd(reinterpret_cast<float4*>(TK) + idx, make_float4(float(T.re), float(T.im), float(K.re), float(K.im)));
}

// ---------------------------------------------------------------------------
// regular (vertex-disjoint) pairs, FP64: one thread per ordered pair
// ---------------------------------------------------------------------------
struct BlockArgs {
  const double* bt_v;
  const double* bt_c;
  const double* bt_area;
  const int32_t* bt_dof;
  const int32_t* bt_vid;
  const int32_t* blk_T;
  const int32_t* blk_N;
  const int64_t* blk_bt_off;
  const int64_t* blk_mat_off;
  const double* k;  // (re, im) per block
  int nblk;
};

__global__ void __launch_bounds__(128) k_regular64(BlockArgs A, const int64_t* __restrict__ cta_prefix,
                                                   double* __restrict__ TK) {
  const int64_t cta = blockIdx.x;
  int lo = 0, hi = A.nblk - 1;
  while (lo < hi) {  // largest i with cta_prefix[i] <= cta
    const int mid = (lo + hi + 1) >> 1;
    if (cta_prefix[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  const int i = lo;
  const int T = A.blk_T[i];
  const int64_t pair = (cta - cta_prefix[i]) * 128 + threadIdx.x;
  if (pair >= int64_t(T) * T) return;
  const int64_t qt = A.blk_bt_off[i] + pair / T;
  const int64_t qs = A.blk_bt_off[i] + pair % T;
  int shared = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) shared += A.bt_vid[3 * qt + a] == A.bt_vid[3 * qs + b];
  if (shared) return;  // singular pairs are handled by k_singular64

  double vt[9], vs[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    vt[c] = A.bt_v[9 * qt + c];
    vs[c] = A.bt_v[9 * qs + c];
  }
  double ot[3], os[3], D[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ot[c] = (vt[c] + vt[3 + c] + vt[6 + c]) * (1.0 / 3.0);
    os[c] = (vs[c] + vs[3 + c] + vs[6 + c]) * (1.0 / 3.0);
    D[c] = ot[c] - os[c];
  }
  const double At2 = 2.0 * A.bt_area[qt], As2 = 2.0 * A.bt_area[qs];
  const double kr = A.k[2 * i], ki = A.k[2 * i + 1];
  double yq[6][3], wq[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
      yq[q][c] = vs[c] + c_tri_s[q] * (vs[3 + c] - vs[c]) + c_tri_t[q] * (vs[6 + c] - vs[c]) - os[c];
    wq[q] = As2 * c_tri_w[q];
  }
  Moments M;
  zero(M);
#pragma unroll 1
  for (int p = 0; p < 6; ++p) {
    double xp[3], e[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xp[c] = vt[c] + c_tri_s[p] * (vt[3 + c] - vt[c]) + c_tri_t[p] * (vt[6 + c] - vt[c]) - ot[c];
      e[c] = xp[c] + D[c];
    }
    const double wp = At2 * c_tri_w[p];
    C2 R{0, 0}, Qp{0, 0}, Ry[3], Qy[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Ry[c] = Qy[c] = C2{0, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double d0 = e[0] - yq[q][0], d1 = e[1] - yq[q][1], d2 = e[2] - yq[q][2];
      const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      C2 G, g;
      helmholtz(kr, ki, r, G, g);
      G = cscale(G, wq[q]);
      g = cscale(g, wq[q]);
      R = cadd(R, G);
      Qp = cadd(Qp, g);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Ry[c] = cadd(Ry[c], cscale(G, yq[q][c]));
        Qy[c] = cadd(Qy[c], cscale(g, yq[q][c]));
      }
    }
    R = cscale(R, wp);
    Qp = cscale(Qp, wp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ry[c] = cscale(Ry[c], wp);
      Qy[c] = cscale(Qy[c], wp);
    }
    M.S0 = cadd(M.S0, R);
    M.Q = cadd(M.Q, Qp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      M.Sx[c] = cadd(M.Sx[c], cscale(R, xp[c]));
      M.Sy[c] = cadd(M.Sy[c], Ry[c]);
      M.Sxy = cadd(M.Sxy, cscale(Ry[c], xp[c]));
      M.Gx[c] = cadd(M.Gx[c], cscale(Qp, xp[c]));
      M.Gy[c] = cadd(M.Gy[c], Qy[c]);
    }
    // C += x' x Qy
    M.C[0] = cadd(M.C[0], csub(cscale(Qy[2], xp[1]), cscale(Qy[1], xp[2])));
    M.C[1] = cadd(M.C[1], csub(cscale(Qy[0], xp[2]), cscale(Qy[2], xp[0])));
    M.C[2] = cadd(M.C[2], csub(cscale(Qy[1], xp[0]), cscale(Qy[0], xp[1])));
  }
  const int N = A.blk_N[i];
  const int64_t base = A.blk_mat_off[i];
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    double pa[3];
    for (int c = 0; c < 3; ++c) pa[c] = vt[3 * a + c] - ot[c];
    const double ca = A.bt_c[3 * qt + a];
    const int m = A.bt_dof[3 * qt + a];
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
      double qb[3];
      for (int c = 0; c < 3; ++c) qb[c] = vs[3 * b + c] - os[c];
      C2 Tv, Kv;
      local_entry(M, pa, qb, D, ca * A.bt_c[3 * qs + b], kr, ki, Tv, Kv);
      add_entry(TK, base + int64_t(m) * N + A.bt_dof[3 * qs + b], Tv, Kv);
    }
  }
}

// ---------------------------------------------------------------------------
// singular pairs (Sauter-Schwab), FP64: one warp per pair
// ---------------------------------------------------------------------------
template <class OutT>
__global__ void __launch_bounds__(256) k_singular64(BlockArgs A, const SingPair* __restrict__ sp,
                                                    int64_t npairs, const double* __restrict__ ss0,
                                                    const double* __restrict__ ss1,
                                                    const double* __restrict__ ss2, int n0, int n1,
                                                    int n2, OutT* __restrict__ TK) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= npairs) return;
  const SingPair P = sp[w];
  const int kind = P.code & 3;
  const int pt0 = (P.code >> 2) & 3, pt1 = (P.code >> 4) & 3, pt2 = (P.code >> 6) & 3;
  const int ps0 = (P.code >> 8) & 3, ps1 = (P.code >> 10) & 3, ps2 = (P.code >> 12) & 3;
  const double* tab = kind == 0 ? ss0 : (kind == 1 ? ss1 : ss2);
  const int npts = kind == 0 ? n0 : (kind == 1 ? n1 : n2);
  const int64_t qt = P.tau, qs = P.sig;
  const double* vt = A.bt_v + 9 * qt;
  const double* vs = A.bt_v + 9 * qs;
  double o[3], e1[3], e2[3], f1[3], f2[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o[c] = vt[3 * pt0 + c];
    e1[c] = vt[3 * pt1 + c] - vt[3 * pt0 + c];
    e2[c] = vt[3 * pt2 + c] - vt[3 * pt1 + c];
    // the trial map shares its origin with the test map (P0 = Q0 for every kind)
    f1[c] = vs[3 * ps1 + c] - vs[3 * ps0 + c];
    f2[c] = vs[3 * ps2 + c] - vs[3 * ps1 + c];
  }
  const double W4 = 4.0 * A.bt_area[qt] * A.bt_area[qs];
  const int i = P.block;
  const double kr = A.k[2 * i], ki = A.k[2 * i + 1];
  Moments M;
  zero(M);
  for (int p = lane; p < npts; p += 32) {
    const double x1 = tab[5 * p], x2 = tab[5 * p + 1], y1 = tab[5 * p + 2], y2 = tab[5 * p + 3];
    const double W = tab[5 * p + 4] * W4;
    double xp[3], yp[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xp[c] = x1 * e1[c] + x2 * e2[c];
      yp[c] = y1 * f1[c] + y2 * f2[c];
    }
    if (kind == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] = (x1 - y1) * e1[c] + (x2 - y2) * e2[c];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] = xp[c] - yp[c];
    }
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    C2 G, g;
    helmholtz(kr, ki, r, G, g);
    G = cscale(G, W);
    g = cscale(g, W);
    M.S0 = cadd(M.S0, G);
    double xy = xp[0] * yp[0] + xp[1] * yp[1] + xp[2] * yp[2];
    M.Sxy = cadd(M.Sxy, cscale(G, xy));
    const double cr[3] = {xp[1] * yp[2] - xp[2] * yp[1], xp[2] * yp[0] - xp[0] * yp[2],
                          xp[0] * yp[1] - xp[1] * yp[0]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      M.Sx[c] = cadd(M.Sx[c], cscale(G, xp[c]));
      M.Sy[c] = cadd(M.Sy[c], cscale(G, yp[c]));
      M.Gx[c] = cadd(M.Gx[c], cscale(g, d[c]));  // only Gx - Gy enters when Delta = 0
      M.C[c] = cadd(M.C[c], cscale(g, cr[c]));
    }
  }
  // warp reduction of the 28 doubles actually used (Q, Gy stay zero)
  double* f = reinterpret_cast<double*>(&M);
  const int nd = sizeof(Moments) / sizeof(double);
#pragma unroll
  for (int q = 0; q < nd; ++q) {
    double v = f[q];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    f[q] = v;
  }
  if (lane < 9) {
    const int a = lane / 3, b = lane % 3;
    double pa[3], qb[3];
    const double D[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pa[c] = vt[3 * a + c] - o[c];
      qb[c] = vs[3 * b + c] - o[c];
    }
    C2 Tv, Kv;
    local_entry(M, pa, qb, D, A.bt_c[3 * qt + a] * A.bt_c[3 * qs + b], kr, ki, Tv, Kv);
    const int N = A.blk_N[i];
    const int64_t ra = A.bt_dof[3 * qt + a], cb = A.bt_dof[3 * qs + b];
    add_entry(TK, A.blk_mat_off[i] + ra * N + cb, Tv, Kv);
    // the swapped pair (sigma, tau) of an adjacent pair: the same value at
    // the transposed position (symmetric Galerkin forms)
    if (kind != 0) add_entry(TK, A.blk_mat_off[i] + cb * N + ra, Tv, Kv);
  }
}

// ---------------------------------------------------------------------------
// transmission Gram values (Eq. 18): one thread per exchange entry
//   G^{ij}[m, n] on triangle t = c_a^i c_b^j int_t n_i . ((x - v_a) x (x - v_b))
// ---------------------------------------------------------------------------
__global__ void k_exchange_values(const XEntry* __restrict__ xe, int64_t nent, const double* __restrict__ bt_v,
                                  const double* __restrict__ bt_c, const double* __restrict__ bt_area,
                                  const int8_t* __restrict__ bt_swap, double* __restrict__ xval) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= nent) return;
  const XEntry X = xe[e];
  const int a = X.ab & 3, b = (X.ab >> 2) & 3;
  const double* v = bt_v + 9 * int64_t(X.bt_i);
  double e1[3], e2[3], n[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = v[3 + c] - v[c];
    e2[c] = v[6 + c] - v[c];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  const double sw = bt_swap[X.bt_i] / nn;
  double acc = 0.0;
  for (int q = 0; q < 6; ++q) {
    double x[3], u[3], w[3];
    for (int c = 0; c < 3; ++c) {
      x[c] = v[c] + c_tri_s[q] * e1[c] + c_tri_t[q] * e2[c];
      u[c] = x[c] - v[3 * a + c];
      w[c] = x[c] - v[3 * b + c];
    }
    const double cr0 = u[1] * w[2] - u[2] * w[1], cr1 = u[2] * w[0] - u[0] * w[2],
                 cr2 = u[0] * w[1] - u[1] * w[0];
    acc += c_tri_w[q] * (n[0] * cr0 + n[1] * cr1 + n[2] * cr2);
  }
  xval[e] = 2.0 * bt_area[X.bt_i] * sw * acc * bt_c[3 * X.bt_i + a] * bt_c[3 * X.bt_j + b];
}

// ---------------------------------------------------------------------------
// incident data (Eq. 22): b_D = 2 int E_inc . psi, b_N = 2 int (d x p) e^{ik0 d.x} . psi
// on Gamma_0 (= -2 <gamma_.,0 E_inc, psi>_x); one thread per (dof of block 0, rhs)
// ---------------------------------------------------------------------------
__global__ void k_rhs(const int32_t* __restrict__ dof_bt, int N0, int nrhs, int64_t n_total,
                      const double* __restrict__ bt_v, const double* __restrict__ bt_c,
                      const double* __restrict__ bt_area, double k0, const double* __restrict__ dirs,
                      const double* __restrict__ pols, double* __restrict__ b) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid >= int64_t(N0) * nrhs) return;
  const int m = int(tid % N0), col = int(tid / N0);
  const double* d = dirs + 3 * col;
  const double* P = pols + 6 * col;  // complex128 x 3
  const C2 p[3] = {{P[0], P[1]}, {P[2], P[3]}, {P[4], P[5]}};
  C2 dxp[3];
  dxp[0] = csub(cscale(p[2], d[1]), cscale(p[1], d[2]));
  dxp[1] = csub(cscale(p[0], d[2]), cscale(p[2], d[0]));
  dxp[2] = csub(cscale(p[1], d[0]), cscale(p[0], d[1]));
  C2 sE{0, 0}, sN{0, 0};
  for (int e = 0; e < 2; ++e) {
    const int code = dof_bt[2 * m + e];
    const int64_t q = code / 3;
    const int a = code % 3;
    const double* v = bt_v + 9 * q;
    const double ca = bt_c[3 * q + a], A2 = 2.0 * bt_area[q];
    for (int qp = 0; qp < 6; ++qp) {
      double x[3], f[3];
      for (int c = 0; c < 3; ++c) {
        x[c] = v[c] + c_tri_s[qp] * (v[3 + c] - v[c]) + c_tri_t[qp] * (v[6 + c] - v[c]);
        f[c] = ca * (x[c] - v[3 * a + c]);
      }
      double sn, cs;
      sincos(k0 * (d[0] * x[0] + d[1] * x[1] + d[2] * x[2]), &sn, &cs);
      const C2 ph{cs * A2 * c_tri_w[qp], sn * A2 * c_tri_w[qp]};
      C2 pe{0, 0}, pn{0, 0};
      for (int c = 0; c < 3; ++c) {
        pe = cadd(pe, cscale(p[c], f[c]));
        pn = cadd(pn, cscale(dxp[c], f[c]));
      }
      sE = cadd(sE, cmul(ph, pe));
      sN = cadd(sN, cmul(ph, pn));
    }
  }
  double* bc = b + 2 * (int64_t(col) * n_total);
  bc[2 * m] = 2.0 * sE.re;
  bc[2 * m + 1] = 2.0 * sE.im;
  bc[2 * (N0 + m)] = 2.0 * sN.re;
  bc[2 * (N0 + m) + 1] = 2.0 * sN.im;
}

// ---------------------------------------------------------------------------
// far field (Stratton-Chu in Omega_0): one CTA per (direction, rhs)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_farfield(const double* __restrict__ x, int64_t n_total, int N0,
                                                  int T0, const double* __restrict__ bt_v,
                                                  const double* __restrict__ bt_c,
                                                  const double* __restrict__ bt_area,
                                                  const int32_t* __restrict__ bt_dof, double k0,
                                                  const double* __restrict__ obs, int nobs,
                                                  double* __restrict__ fout) {
  const int o = blockIdx.x, col = blockIdx.y;
  const double xh[3] = {obs[3 * o], obs[3 * o + 1], obs[3 * o + 2]};
  const double* xc = x + 2 * int64_t(col) * n_total;
  double acc[12];
  for (int c = 0; c < 12; ++c) acc[c] = 0.0;  // wa (re,im)x3, wb (re,im)x3
  for (int it = threadIdx.x; it < T0 * 6; it += blockDim.x) {
    const int q = it / 6, qp = it % 6;
    const double* v = bt_v + 9 * int64_t(q);
    double y[3];
    for (int c = 0; c < 3; ++c) y[c] = v[c] + c_tri_s[qp] * (v[3 + c] - v[c]) + c_tri_t[qp] * (v[6 + c] - v[c]);
    double sn, cs;
    sincos(-k0 * (xh[0] * y[0] + xh[1] * y[1] + xh[2] * y[2]), &sn, &cs);
    const double w = 2.0 * bt_area[q] * c_tri_w[qp];
    for (int a = 0; a < 3; ++a) {
      const int m = bt_dof[3 * q + a];
      const double ca = bt_c[3 * q + a] * w;
      const C2 uD{xc[2 * m], xc[2 * m + 1]}, uN{xc[2 * (N0 + m)], xc[2 * (N0 + m) + 1]};
      const C2 fD = cmul(uD, C2{cs * ca, sn * ca}), fN = cmul(uN, C2{cs * ca, sn * ca});
      for (int c = 0; c < 3; ++c) {
        const double f = y[c] - v[3 * a + c];
        acc[2 * c] += fD.re * f;
        acc[2 * c + 1] += fD.im * f;
        acc[6 + 2 * c] += fN.re * f;
        acc[6 + 2 * c + 1] += fN.im * f;
      }
    }
  }
  __shared__ double red[8][12];
  for (int c = 0; c < 12; ++c) {
    double v = acc[c];
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    acc[c] = v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int c = 0; c < 12; ++c) red[warp][c] = acc[c];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[12];
    for (int c = 0; c < 12; ++c) {
      s[c] = 0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) s[c] += red[w][c];
    }
    // E = i k0/(4 pi) [xh x wa + (xh x wb) x xh]
    double out[6];
    for (int ri = 0; ri < 2; ++ri) {
      const double wa[3] = {s[ri], s[2 + ri], s[4 + ri]};
      const double wb[3] = {s[6 + ri], s[8 + ri], s[10 + ri]};
      const double t1[3] = {xh[1] * wa[2] - xh[2] * wa[1], xh[2] * wa[0] - xh[0] * wa[2],
                            xh[0] * wa[1] - xh[1] * wa[0]};
      const double u[3] = {xh[1] * wb[2] - xh[2] * wb[1], xh[2] * wb[0] - xh[0] * wb[2],
                           xh[0] * wb[1] - xh[1] * wb[0]};
      const double t2[3] = {u[1] * xh[2] - u[2] * xh[1], u[2] * xh[0] - u[0] * xh[2],
                            u[0] * xh[1] - u[1] * xh[0]};
      for (int c = 0; c < 3; ++c) out[2 * c + ri] = t1[c] + t2[c];
    }
    double* f = fout + 2 * 3 * (int64_t(col) * nobs + o);
    const double sc = k0 * INV_FOUR_PI;
    for (int c = 0; c < 3; ++c) {  // multiply by i sc
      f[2 * c] = -sc * out[2 * c + 1];
      f[2 * c + 1] = sc * out[2 * c];
    }
  }
}

template <class MatT>
__global__ void k_split_block(const MatT* __restrict__ TK, int64_t n, double* __restrict__ T,
                              double* __restrict__ K) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n) return;
  T[2 * e] = TK[4 * e];
  T[2 * e + 1] = TK[4 * e + 1];
  K[2 * e] = TK[4 * e + 2];
  K[2 * e + 1] = TK[4 * e + 3];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static void upload_rule_constants(cudaStream_t s) {
  const TriRule& r = triangle_rule6();
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_tri_s, r.s, sizeof(r.s), 0, cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_tri_t, r.t, sizeof(r.t), 0, cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_tri_w, r.w, sizeof(r.w), 0, cudaMemcpyHostToDevice, s));
}

static BlockArgs block_args(mtf_system sys) {
  mtf_mesh m = sys->mesh;
  BlockArgs A;
  A.bt_v = m->d_bt_v.p;
  A.bt_c = m->d_bt_c.p;
  A.bt_area = m->d_bt_area.p;
  A.bt_dof = m->d_bt_dof.p;
  A.bt_vid = m->d_bt_vid.p;
  A.blk_T = m->d_blk_T.p;
  A.blk_N = m->d_blk_N.p;
  A.blk_bt_off = m->d_blk_bt_off.p;
  A.blk_mat_off = m->d_blk_mat_off.p;
  A.k = sys->d_k.p;
  A.nblk = m->nd;
  return A;
}

// v[k] -> out[k] = fl(v[k]), out[n + k] = fl(v[k] - fl(v[k]))
__global__ void k_split_pairs(const double* __restrict__ v, int64_t n, float* __restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double a = v[t];
  const float h = float(a);
  out[t] = h;
  out[n + t] = float(a - double(h));
}

void launch_assemble(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  upload_rule_constants(s);
  // Sauter-Schwab tables (once per system)
  if (sys->ss_npts[0] == 0) {
    for (int kind = 0; kind < 3; ++kind) {
      std::vector<double> pts;
      sauter_schwab_rule(kind, sys->opt.n_ss, pts);
      sys->d_ss_pts[kind].upload(pts, s);
      MTF_CUDA(cudaStreamSynchronize(s));
      sys->ss_npts[kind] = int(pts.size() / 5);
    }
  }
  BlockArgs A = block_args(sys);
  const int64_t np = int64_t(m->sing.size());
  const unsigned sblocks = unsigned((np * 32 + 255) / 256);
  const bool fp64_blocks = sys->opt.precision == MTF_PREC_FP64 || sys->opt.residual_fp64;
  if (fp64_blocks) {
    sys->d_TK64.alloc(size_t(m->n_mat) * 4);
    MTF_CUDA(cudaMemsetAsync(sys->d_TK64.p, 0, size_t(m->n_mat) * 4 * sizeof(double), s));
    const int64_t nct = m->reg_cta_prefix.back();
    if (nct > 0)
      MTF_LAUNCH(KID_REGULAR64, s, k_regular64<<<unsigned(nct), 128, 0, s>>>(A, m->d_reg_cta_prefix.p, sys->d_TK64.p));
    if (np > 0)
      MTF_LAUNCH(KID_SINGULAR64, s, k_singular64<double><<<sblocks, 256, 0, s>>>(
          A, m->d_sing.p, np, sys->d_ss_pts[0].p, sys->d_ss_pts[1].p, sys->d_ss_pts[2].p, sys->ss_npts[0],
          sys->ss_npts[1], sys->ss_npts[2], sys->d_TK64.p));
  }
  if (fp64_blocks && sys->opt.precision != MTF_PREC_FP64) {
    // residual_fp64: the FP64 entries split into FP32 pairs once per assembly,
    // for the double-float residual matvec
    const int64_t nv = m->n_mat * 4;
    sys->d_TK64hl.alloc(size_t(nv) * 2);
    MTF_LAUNCH(KID_MISC, s, k_split_pairs<<<unsigned((nv + 255) / 256), 256, 0, s>>>(sys->d_TK64.p, nv,
                                                                                     sys->d_TK64hl.p));
  }
  if (sys->opt.precision != MTF_PREC_FP64) {
    // mixed: FP32 storage; regular pairs in FP32, singular pairs in FP64
    sys->d_TK32.alloc(size_t(m->n_mat) * 4);
    MTF_CUDA(cudaMemsetAsync(sys->d_TK32.p, 0, size_t(m->n_mat) * 4 * sizeof(float), s));
    launch_assemble_regular32(sys, s);
    if (np > 0)
      MTF_LAUNCH(KID_SINGULAR64, s, k_singular64<float><<<sblocks, 256, 0, s>>>(
          A, m->d_sing.p, np, sys->d_ss_pts[0].p, sys->d_ss_pts[1].p, sys->d_ss_pts[2].p, sys->ss_npts[0],
          sys->ss_npts[1], sys->ss_npts[2], sys->d_TK32.p));
    if (sys->opt.mv_tensor) tc_build_operator(sys, s);
    else tile_matvec_operator(sys, s);
  }
  launch_exchange_values(sys, s);
}

__global__ void k_d2f(const double* __restrict__ a, int64_t n, float* __restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) out[t] = float(a[t]);
}

void launch_exchange_values(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const int64_t nent = m->n_rows * 6;
  sys->d_xval.alloc(size_t(nent));
  MTF_LAUNCH(KID_XVALUES, s, k_exchange_values<<<unsigned((nent + 255) / 256), 256, 0, s>>>(
      m->d_xent.p, nent, m->d_bt_v.p, m->d_bt_c.p, m->d_bt_area.p, m->d_bt_swap.p, sys->d_xval.p));
  // FP32 copy for the FP32 epilogues of the mixed inner solver
  sys->d_xval32.alloc(size_t(nent));
  MTF_LAUNCH(KID_XVALUES, s, k_d2f<<<unsigned((nent + 255) / 256), 256, 0, s>>>(sys->d_xval.p, nent, sys->d_xval32.p));
}

void launch_rhs(mtf_system sys, int nrhs, const double* d_dirs, const double* d_pols, double* b,
                cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  upload_rule_constants(s);
  MTF_CUDA(cudaMemsetAsync(b, 0, size_t(m->n_total) * nrhs * 2 * sizeof(double), s));
  const int N0 = m->blk[0].N;
  const int64_t nth = int64_t(N0) * nrhs;
  MTF_LAUNCH(KID_RHS, s, k_rhs<<<unsigned((nth + 127) / 128), 128, 0, s>>>(m->d_dof_bt.p, N0, nrhs, m->n_total, m->d_bt_v.p,
                                                      m->d_bt_c.p, m->d_bt_area.p, sys->k0, d_dirs, d_pols, b));
  MTF_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// near field (Stratton-Chu, Eq. 8): for a point x in Omega_i,
//   U(x) = H_k(a)(x) + E_k(b)(x),  a = gamma_D U,  b = gamma_N U (N slot / rho_i),
//   H_k a = int grad_x G x a,  E_k b = i k int G b - 1/(i k) int grad_x G div b,
// with k = k_i, the RWG fields of block i's coefficients and div psi_a = 2 c_a.
// One CTA per (point, rhs); the 6-point rule on every triangle of block i.
// blk: per block {first block-triangle, triangles, N, dof offset}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_nearfield(const double* __restrict__ x, int64_t n_total,
                                                   const double* __restrict__ bt_v,
                                                   const double* __restrict__ bt_c,
                                                   const double* __restrict__ bt_area,
                                                   const int32_t* __restrict__ bt_dof,
                                                   const int64_t* __restrict__ blk, const double* __restrict__ kk,
                                                   const double* __restrict__ rho, const double* __restrict__ pts,
                                                   const int32_t* __restrict__ dom, int npts,
                                                   double* __restrict__ fout) {
  const int p = blockIdx.x, col = blockIdx.y;
  const int i = dom[p];
  const double X[3] = {pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]};
  const int64_t q0 = blk[4 * i], T = blk[4 * i + 1], N = blk[4 * i + 2], off = blk[4 * i + 3];
  const double kr = kk[2 * i], ki = kk[2 * i + 1];
  const double rr = rho[2 * i], ri = rho[2 * i + 1], rn = rr * rr + ri * ri;
  const C2 irho{rr / rn, -ri / rn};
  const C2 ik{-ki, kr};
  const double kn = kr * kr + ki * ki;
  const C2 minv_ik{ki / kn, kr / kn};  // -1 / (i k)
  const double* xc = x + 2 * int64_t(col) * n_total;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t it = threadIdx.x; it < T * 6; it += blockDim.x) {
    const int64_t q = q0 + it / 6;
    const int qp = int(it % 6);
    const double* v = bt_v + 9 * q;
    double y[3], d[3];
    for (int c = 0; c < 3; ++c) {
      y[c] = v[c] + c_tri_s[qp] * (v[3 + c] - v[c]) + c_tri_t[qp] * (v[6 + c] - v[c]);
      d[c] = X[c] - y[c];
    }
    const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    C2 G, g;
    helmholtz(kr, ki, R, G, g);  // grad_x G = g d
    const double w = 2.0 * bt_area[q] * c_tri_w[qp];
    C2 av[3] = {{0, 0}, {0, 0}, {0, 0}}, bv[3] = {{0, 0}, {0, 0}, {0, 0}}, divb{0, 0};
    for (int a = 0; a < 3; ++a) {
      const int64_t m = bt_dof[3 * q + a];
      const double ca = bt_c[3 * q + a];
      const C2 uD{xc[2 * (off + m)], xc[2 * (off + m) + 1]};
      const C2 uN = cmul(C2{xc[2 * (off + N + m)], xc[2 * (off + N + m) + 1]}, irho);
      for (int c = 0; c < 3; ++c) {
        const double f = ca * (y[c] - v[3 * a + c]);
        av[c] = cadd(av[c], cscale(uD, f));
        bv[c] = cadd(bv[c], cscale(uN, f));
      }
      divb = cadd(divb, cscale(uN, 2.0 * ca));
    }
    const C2 ikG = cmul(ik, G);
    const C2 e2 = cmul(minv_ik, cmul(g, divb));
    for (int c = 0; c < 3; ++c) {
      const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      const C2 cr = csub(cscale(av[c2], d[c1]), cscale(av[c1], d[c2]));  // (d x a)_c
      const C2 e = cadd(cadd(cmul(g, cr), cmul(ikG, bv[c])), cscale(e2, d[c]));
      acc[2 * c] += w * e.re;
      acc[2 * c + 1] += w * e.im;
    }
  }
  __shared__ double red[8][6];
  for (int c = 0; c < 6; ++c) {
    double v = acc[c];
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    acc[c] = v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int c = 0; c < 6; ++c) red[warp][c] = acc[c];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0;
    for (int wi = 0; wi < int(blockDim.x >> 5); ++wi) t += red[wi][threadIdx.x];
    fout[(int64_t(col) * npts + p) * 6 + threadIdx.x] = t;
  }
}

void launch_nearfield(mtf_system sys, const double* x, int nrhs, const double* d_pts, const int32_t* d_dom,
                      int npts, double* f, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  upload_rule_constants(s);
  std::vector<int64_t> blk(static_cast<size_t>(4 * m->nd));
  for (int i = 0; i < m->nd; ++i) {
    blk[size_t(4 * i)] = m->blk[i].bt_off;
    blk[size_t(4 * i + 1)] = m->blk[i].T;
    blk[size_t(4 * i + 2)] = m->blk[i].N;
    blk[size_t(4 * i + 3)] = m->blk[i].dof_off;
  }
  DevBuf<int64_t> d_blk;
  d_blk.upload(blk, s);
  MTF_LAUNCH(KID_FARFIELD, s, k_nearfield<<<dim3(unsigned(npts), unsigned(nrhs)), 256, 0, s>>>(
      x, m->n_total, m->d_bt_v.p, m->d_bt_c.p, m->d_bt_area.p, m->d_bt_dof.p, d_blk.p, sys->d_k.p, sys->d_rho.p,
      d_pts, d_dom, npts, f));
  MTF_CUDA(cudaStreamSynchronize(s));  // d_blk is released on return
}

void launch_farfield(mtf_system sys, const double* x, int nrhs, const double* d_obs, int nobs, double* f,
                     cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  upload_rule_constants(s);
  dim3 grid{unsigned(nobs), unsigned(nrhs), 1u};
  MTF_LAUNCH(KID_FARFIELD, s, k_farfield<<<grid, 256, 0, s>>>(x, m->n_total, m->blk[0].N, m->blk[0].T, m->d_bt_v.p, m->d_bt_c.p,
                                   m->d_bt_area.p, m->d_bt_dof.p, sys->k0, d_obs, nobs, f));
  MTF_CUDA(cudaGetLastError());
}

void launch_get_block(mtf_system sys, int i, double* t_out, double* k_out, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const int64_t n = int64_t(m->blk[i].N) * m->blk[i].N;
  if (sys->opt.precision == MTF_PREC_FP64) {
    const double* src = sys->d_TK64.p + 4 * m->blk[i].mat_off;
    MTF_LAUNCH(KID_SPLIT, s, k_split_block<double><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, n, t_out, k_out));
  } else {
    const float* src = sys->d_TK32.p + 4 * m->blk[i].mat_off;
    MTF_LAUNCH(KID_SPLIT, s, k_split_block<float><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, n, t_out, k_out));
  }
  MTF_CUDA(cudaGetLastError());
}

}  // namespace mtf
