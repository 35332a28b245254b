// Mixed-precision assembly of the regular (vertex-disjoint) triangle pairs.
//
// Same Galerkin integrals as k_regular64 (Eqs. 7-9 tested with Eq. 5), with
// the Helmholtz kernel evaluated in FP32 except for the part of the phase
// that FP32 cannot carry.  With centroids o_tau, o_sigma (FP64), Delta =
// o_tau - o_sigma, R0 = |Delta|, every point pair has r = R0 + dr with
//   dr = (2 Delta.e + e.e) / (r + R0),   e = x' - y'  (local offsets),
// which is free of cancellation, and
//   exp(i k r) = exp(i k R0) exp(i k dr).
// The per-pair factor exp(i k R0) is formed from an FP64 phase reduced modulo
// 2 pi, the per-point factor exp(i k dr) from the Taylor series of sin and cos
// (|k dr| is bounded by k times the pair's extent; larger arguments fall back
// to sincosf).  Kernel sums are accumulated in FP32 and rotated by
// exp(i k R0) once per pair.  Absolute phase errors stay near the FP32
// rounding of the factors (~1e-7) instead of k r 2^-24.
#include <cmath>

#include "common.h"

namespace mtf {

// the 6-point rule (own copy in this translation unit)
__constant__ double c_tri_s[6], c_tri_t[6], c_tri_w[6];

#define INV_FOUR_PI_F 0.0795774715459476679f
#define TWO_PI_D 6.283185307179586476925
#define INV_TWO_PI_D 0.159154943091895335769

struct F2 {
  float re, im;
};
__device__ __forceinline__ F2 fmul(F2 a, F2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ F2 fsc(F2 a, float s) { return {a.re * s, a.im * s}; }
__device__ __forceinline__ F2 fadd(F2 a, F2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ F2 fsub(F2 a, F2 b) { return {a.re - b.re, a.im - b.im}; }

// sin and cos from their Taylor series (coefficients (-1)^j / (2j+1)! and
// (-1)^j / (2j)!); truncation error below 1e-9 for |x| <= 1.6.
__device__ __forceinline__ void sincos_taylor(float x, float* s, float* c) {
  const float x2 = x * x;
  // sin = x - x^3/3! + x^5/5! - x^7/7! + x^9/9! - x^11/11! + x^13/13!
  float s_ = 1.0f / 6227020800.0f;
  s_ = fmaf(s_, x2, -1.0f / 39916800.0f);
  s_ = fmaf(s_, x2, 1.0f / 362880.0f);
  s_ = fmaf(s_, x2, -1.0f / 5040.0f);
  s_ = fmaf(s_, x2, 1.0f / 120.0f);
  s_ = fmaf(s_, x2, -1.0f / 6.0f);
  s_ = s_ * x2;
  *s = fmaf(s_, x, x);
  // cos = 1 - x^2/2! + x^4/4! - x^6/6! + x^8/8! - x^10/10! + x^12/12! - x^14/14!
  float c_ = -1.0f / 87178291200.0f;
  c_ = fmaf(c_, x2, 1.0f / 479001600.0f);
  c_ = fmaf(c_, x2, -1.0f / 3628800.0f);
  c_ = fmaf(c_, x2, 1.0f / 40320.0f);
  c_ = fmaf(c_, x2, -1.0f / 720.0f);
  c_ = fmaf(c_, x2, 1.0f / 24.0f);
  c_ = fmaf(c_, x2, -0.5f);
  *c = fmaf(c_, x2, 1.0f);
}

// Per block-triangle FP32 geometry relative to the centroid (FP64):
// quadrature points (6x3), weights 2A w (6), vertices (3x3), RWG c_a (3).
struct Geom32Args {
  const double* bt_v;
  const double* bt_c;
  const double* bt_area;
  int64_t n_bt;
  double* cen;   // 3 per bt
  float* qx;     // 18 per bt
  float* qw;     // 6 per bt
  float* pv;     // 9 per bt
  float* cc;     // 3 per bt
};

__global__ void k_geom32(Geom32Args G) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= G.n_bt) return;
  const double* v = G.bt_v + 9 * q;
  double o[3];
  for (int c = 0; c < 3; ++c) o[c] = (v[c] + v[3 + c] + v[6 + c]) * (1.0 / 3.0);
  for (int c = 0; c < 3; ++c) G.cen[3 * q + c] = o[c];
  for (int p = 0; p < 6; ++p) {
    for (int c = 0; c < 3; ++c)
      G.qx[18 * q + 3 * p + c] =
          float(v[c] - o[c] + c_tri_s[p] * (v[3 + c] - v[c]) + c_tri_t[p] * (v[6 + c] - v[c]));
    G.qw[6 * q + p] = float(2.0 * G.bt_area[q] * c_tri_w[p]);
  }
  for (int a = 0; a < 3; ++a) {
    for (int c = 0; c < 3; ++c) G.pv[9 * q + 3 * a + c] = float(v[3 * a + c] - o[c]);
    G.cc[3 * q + a] = float(G.bt_c[3 * q + a]);
  }
}

struct Reg32Args {
  const double* cen;
  const float* qx;
  const float* qw;
  const float* pv;
  const float* cc;
  const int32_t* bt_dof;
  const int32_t* bt_vid;
  const int32_t* blk_T;
  const int32_t* blk_N;
  const int64_t* blk_bt_off;
  const int64_t* blk_mat_off;
  const double* k;
  int nblk;
};

__global__ void __launch_bounds__(128) k_regular32(Reg32Args A, const int64_t* __restrict__ cta_prefix,
                                                   float* __restrict__ TK) {
  const int64_t cta = blockIdx.x;
  int lo = 0, hi = A.nblk - 1;
  while (lo < hi) {
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
  if (shared) return;

  // ---- FP64 per-pair part: Delta, R0, exp(i k R0) ------------------------
  const double kr = A.k[2 * i];
  const double dD0 = A.cen[3 * qt] - A.cen[3 * qs];
  const double dD1 = A.cen[3 * qt + 1] - A.cen[3 * qs + 1];
  const double dD2 = A.cen[3 * qt + 2] - A.cen[3 * qs + 2];
  const double R2 = dD0 * dD0 + dD1 * dD1 + dD2 * dD2;
  const float R0f = sqrtf(float(R2));
  const double R0 = double(R0f) + (R2 - double(R0f) * double(R0f)) * double(0.5f / R0f);
  const double ph = kr * R0;
  const double phr = ph - TWO_PI_D * rint(ph * INV_TWO_PI_D);
  float s0, c0;
  sincosf(float(phr), &s0, &c0);
  const float D[3] = {float(dD0), float(dD1), float(dD2)};
  const float R0s = float(R0);
  const float k = float(kr);

  float yq[6][3], wq[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
#pragma unroll
    for (int c = 0; c < 3; ++c) yq[q][c] = A.qx[18 * qs + 3 * q + c];
    wq[q] = A.qw[6 * qs + q];
  }
  F2 S0{0, 0}, Sxy{0, 0}, Q{0, 0}, Sx[3], Sy[3], Gx[3], Gy[3], C[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) Sx[c] = Sy[c] = Gx[c] = Gy[c] = C[c] = F2{0, 0};
#pragma unroll 1
  for (int p = 0; p < 6; ++p) {
    float xp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) xp[c] = A.qx[18 * qt + 3 * p + c];
    const float wp = A.qw[6 * qt + p];
    F2 R{0, 0}, Qp{0, 0}, Ry[3], Qy[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Ry[c] = Qy[c] = F2{0, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const float e0 = xp[0] - yq[q][0], e1 = xp[1] - yq[q][1], e2 = xp[2] - yq[q][2];
      const float u = fmaf(2.0f * D[0] + e0, e0, fmaf(2.0f * D[1] + e1, e1, (2.0f * D[2] + e2) * e2));
      const float t2 = R0s * R0s + u;              // r^2
      const float rinv = rsqrtf(t2);
      const float r = t2 * rinv;
      const float dr = u / (r + R0s);
      const float arg = k * dr;
      float sn, cs;
      if (fabsf(arg) <= 1.6f) sincos_taylor(arg, &sn, &cs);
      else sincosf(arg, &sn, &cs);
      const float amp = INV_FOUR_PI_F * rinv;
      F2 G{amp * cs, amp * sn};                    // exp(i k dr) / (4 pi r)
      // g = G (i k - 1/r) / r
      F2 g{(-rinv * G.re - k * G.im) * rinv, (k * G.re - rinv * G.im) * rinv};
      G = fsc(G, wq[q]);
      g = fsc(g, wq[q]);
      R = fadd(R, G);
      Qp = fadd(Qp, g);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Ry[c] = fadd(Ry[c], fsc(G, yq[q][c]));
        Qy[c] = fadd(Qy[c], fsc(g, yq[q][c]));
      }
    }
    R = fsc(R, wp);
    Qp = fsc(Qp, wp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ry[c] = fsc(Ry[c], wp);
      Qy[c] = fsc(Qy[c], wp);
    }
    S0 = fadd(S0, R);
    Q = fadd(Q, Qp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Sx[c] = fadd(Sx[c], fsc(R, xp[c]));
      Sy[c] = fadd(Sy[c], Ry[c]);
      Sxy = fadd(Sxy, fsc(Ry[c], xp[c]));
      Gx[c] = fadd(Gx[c], fsc(Qp, xp[c]));
      Gy[c] = fadd(Gy[c], Qy[c]);
    }
    C[0] = fadd(C[0], fsub(fsc(Qy[2], xp[1]), fsc(Qy[1], xp[2])));
    C[1] = fadd(C[1], fsub(fsc(Qy[0], xp[2]), fsc(Qy[2], xp[0])));
    C[2] = fadd(C[2], fsub(fsc(Qy[1], xp[0]), fsc(Qy[0], xp[1])));
  }
  // rotate every moment by exp(i k R0)
  const F2 e0{c0, s0};
  S0 = fmul(S0, e0);
  Sxy = fmul(Sxy, e0);
  Q = fmul(Q, e0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Sx[c] = fmul(Sx[c], e0);
    Sy[c] = fmul(Sy[c], e0);
    Gx[c] = fmul(Gx[c], e0);
    Gy[c] = fmul(Gy[c], e0);
    C[c] = fmul(C[c], e0);
  }
  // T_ab = c_a c_b [ -ik (Sxy - q'.Sx - p'.Sy + (p'.q') S0) - 4/(ik) S0 ]
  // K_ab = -c_a c_b [ (q'-p'-D).C - p'.(D x Gy) - q'.(Gx x D) + (q' x p').(Gx - Gy + D Q) ]
  F2 DxGy[3], GxxD[3], Dm[3];
  DxGy[0] = fsub(fsc(Gy[2], D[1]), fsc(Gy[1], D[2]));
  DxGy[1] = fsub(fsc(Gy[0], D[2]), fsc(Gy[2], D[0]));
  DxGy[2] = fsub(fsc(Gy[1], D[0]), fsc(Gy[0], D[1]));
  GxxD[0] = fsub(fsc(Gx[1], D[2]), fsc(Gx[2], D[1]));
  GxxD[1] = fsub(fsc(Gx[2], D[0]), fsc(Gx[0], D[2]));
  GxxD[2] = fsub(fsc(Gx[0], D[1]), fsc(Gx[1], D[0]));
#pragma unroll
  for (int c = 0; c < 3; ++c) Dm[c] = fadd(fsub(Gx[c], Gy[c]), fsc(Q, D[c]));
  const float inv4k = 4.0f / k;
  const int N = A.blk_N[i];
  const int64_t base = A.blk_mat_off[i];
#pragma unroll 1
  for (int a = 0; a < 3; ++a) {
    const float pa[3] = {A.pv[9 * qt + 3 * a], A.pv[9 * qt + 3 * a + 1], A.pv[9 * qt + 3 * a + 2]};
    const float ca = A.cc[3 * qt + a];
    const int m = A.bt_dof[3 * qt + a];
    // parts depending on a only
    F2 Xa = Sxy;
    F2 Ka{0, 0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Xa = fsub(Xa, fsc(Sy[c], pa[c]));
      Ka = fsub(Ka, fadd(fsc(C[c], pa[c] + D[c]), fsc(DxGy[c], pa[c])));
    }
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
      const float qb[3] = {A.pv[9 * qs + 3 * b], A.pv[9 * qs + 3 * b + 1], A.pv[9 * qs + 3 * b + 2]};
      const float cab = ca * A.cc[3 * qs + b];
      F2 X = Xa;
      F2 Ks = Ka;
      const float pq = pa[0] * qb[0] + pa[1] * qb[1] + pa[2] * qb[2];
      const float qxp[3] = {qb[1] * pa[2] - qb[2] * pa[1], qb[2] * pa[0] - qb[0] * pa[2],
                            qb[0] * pa[1] - qb[1] * pa[0]};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        X = fsub(X, fsc(Sx[c], qb[c]));
        Ks = fadd(Ks, fsub(fsc(C[c], qb[c]), fsc(GxxD[c], qb[c])));
        Ks = fadd(Ks, fsc(Dm[c], qxp[c]));
      }
      X = fadd(X, fsc(S0, pq));
      // -ik X + (4i/k) S0
      const F2 Tv{cab * (k * X.im - inv4k * S0.im), cab * (-k * X.re + inv4k * S0.re)};
      const F2 Kv = fsc(Ks, -cab);
      float4* e = reinterpret_cast<float4*>(TK) + base + int64_t(m) * N + A.bt_dof[3 * qs + b];
      atomicAdd(e, make_float4(Tv.re, Tv.im, Kv.re, Kv.im));
    }
  }
}

void launch_assemble_regular32(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const TriRule& rule = triangle_rule6();
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_tri_s, rule.s, sizeof(rule.s), 0, cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_tri_t, rule.t, sizeof(rule.t), 0, cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_tri_w, rule.w, sizeof(rule.w), 0, cudaMemcpyHostToDevice, s));
  if (!sys->d_cen.p) {
    sys->d_cen.alloc(size_t(m->n_bt) * 3);
    sys->d_qx.alloc(size_t(m->n_bt) * 18);
    sys->d_qw.alloc(size_t(m->n_bt) * 6);
    sys->d_pv.alloc(size_t(m->n_bt) * 9);
    sys->d_cc.alloc(size_t(m->n_bt) * 3);
  }
  Geom32Args G{m->d_bt_v.p, m->d_bt_c.p, m->d_bt_area.p, m->n_bt,
               sys->d_cen.p, sys->d_qx.p, sys->d_qw.p, sys->d_pv.p, sys->d_cc.p};
  MTF_LAUNCH(KID_MISC, s, k_geom32<<<unsigned((m->n_bt + 127) / 128), 128, 0, s>>>(G));
  Reg32Args A{sys->d_cen.p, sys->d_qx.p, sys->d_qw.p, sys->d_pv.p, sys->d_cc.p, m->d_bt_dof.p, m->d_bt_vid.p,
              m->d_blk_T.p, m->d_blk_N.p, m->d_blk_bt_off.p, m->d_blk_mat_off.p, sys->d_k.p, m->nd};
  const int64_t nct = m->reg_cta_prefix.back();
  if (nct > 0)
    MTF_LAUNCH(KID_REGULAR32, s, k_regular32<<<unsigned(nct), 128, 0, s>>>(A, m->d_reg_cta_prefix.p, sys->d_TK32.p));
}

}  // namespace mtf
