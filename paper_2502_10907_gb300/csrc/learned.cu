// Learned correction of the block-OSRC preconditioner (not in the paper).
//
// The preconditioner stays linear in r:  z = P r + C r,  P the block-OSRC
// operator and C a local stencil.  For dof m of block i and the 4 RWG
// neighbours of m (the other edges of its two triangles on Gamma_i,
// ascending local index) -- stencil slots q = 0 (m itself) .. 4 -- and the
// two sources s in {r, P r},
//   (C r)_D[m] = sum_{q,s} a[q,s,DD] s_D[q] + a[q,s,DN] s_N[q]
//   (C r)_N[m] = sum_{q,s} a[q,s,ND] s_D[q] + a[q,s,NN] s_N[q]
// with complex coefficients a, kLO = 80 reals per dof ordered
// [q][s][DD, DN, ND, NN][re, im].  Two parametrisations of a:
//  * table: the coefficients themselves are the trainable parameters
//    (kLO x n_rows, feature-major);
//  * network: a[m] = g(x_m), g a two-hidden-layer ReLU network of kLF = 10
//    geometric features of the dof (k_i l_m, rho_i, exterior flag, k_i l of
//    the 4 neighbours, k_i^2 (A_1 + A_2) of its two triangles, the cosine
//    between their normals, junction flag); parameters are augmented
//    matrices [W | b] row-major, layer after layer (W1 kLH x 11, W2 kLH x
//    (kLH+1), W3 80 x (kLH+1)).
// Both start at zero output, i.e. at plain block-OSRC.
//
// Training objective (power loss): with c0 the mean Rayleigh quotient
// <z, M P z> / <z, z> of the plain preconditioned operator over random z
// and E = I - M (P + C) / c0 the error propagator of Richardson's iteration
// with step 1 / c0,
//     L = mean_z ||E^K z||^2 / ||z||^2
// over complex Rademacher vectors z (counter-based SplitMix64 draws).  It
// estimates sum_i |1 - lambda_i / c0|^(2K) over the eigenvalues of
// M (P + C), which grows with every eigenvalue outside the disc
// |lambda - c0| < |c0| (the outliers that slow restarted GMRES) and
// ignores the well-clustered ones.  The gradient back-propagates through
// the K steps: a_K = 2 e_K / (||z||^2 batch), b = M^H a_{j+1},
// dL/da (stencil coefficients) += (-b / conj(c0)) conj(source of step j),
// a_j = a_{j+1} - (P^H (b + C_P^H b) + C_r^H b) / conj(c0), with C_r and C_P
// the parts of C acting on r and on P r.  All vectors are complex64 and all
// operators the FP32 kernels of the inner solver.
//
// Network activations are stored feature-major (value f of row q at
// [f * ld + q]).  Every layer of the network -- forward, the backward
// products and the weight gradients -- is a matrix product on the tensor
// cores (tc_gemm.cu: FP16 hi + lo operands, FP32 accumulation), with the
// bias folded in as a column (row) of ones and ReLU or its derivative in the
// product's epilogue.
#include <algorithm>
#include <cmath>
#include <random>

#include "common.h"
#include "tc_gemm.h"

namespace mtf {

constexpr int kLF = 10;  // geometric features
constexpr int kLO = 80;  // stencil coefficients (re, im)
constexpr int kLH = 256;  // hidden width
constexpr int kLW1 = kLH * (kLF + 1), kLW2 = kLH * (kLH + 1), kLW3 = kLO * (kLH + 1);
constexpr int kLNetParams = kLW1 + kLW2 + kLW3;
constexpr int kLMaxBatch = 32;
constexpr int kLMaxK = 16;

struct LearnedState {
  int kind = MTF_LEARNED_TABLE;
  int64_t nparam = 0;
  DevBuf<float> params, grad, am, av;  // table: params is the coefficient table
  int64_t adam_t = 0;
  DevBuf<int32_t> nbr;   // 4 global rows per global dof row
  DevBuf<int32_t> slot;  // slot of row g in the stencil of its k-th neighbour (1..4)
  DevBuf<float> X;       // geometric features, kLF x n_rows
  DevBuf<float> coef;    // network: stencil coefficients of the current parameters, kLO x n_rows
  // network scratch (ld = rows) and the coefficient gradient G3 (kLO x rows)
  DevBuf<float> H1, H2, Y, G3, G2, G1;
  int64_t rows_cap = 0;
  // power-loss scratch (complex64 columns of n_total)
  DevBuf<float> Zb, E, PE, T, MT, A, B, CRH, CPH, U, CA;
  DevBuf<double> acc;
  TcGemm* gemm = nullptr;  // tensor-core products of the network
  uint64_t draws = 0;    // random vectors drawn so far (counter of the generator)
  bool centred = false;
  double center_re = 1.0, center_im = 0.0;
};

void destroy_learned(LearnedState* l) {
  if (l) tg_destroy(l->gemm);
  delete l;
}

static inline unsigned nbk(int64_t n, int t) { return unsigned((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// out[c] += sum_k |v^c[k]|^2 over n complex entries (column stride ld)
__global__ void __launch_bounds__(256) k_l_sumsq(const float* __restrict__ v, int64_t ld, int64_t n,
                                                 double* __restrict__ out) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float a = 0.f;
  if (k < n) {
    const float2 x = reinterpret_cast<const float2*>(v + 2 * int64_t(c) * ld)[k];
    a = x.x * x.x + x.y * x.y;
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out + c, double(a));
}

// out[2c], out[2c+1] += sum_k conj(a^c[k]) b^c[k]
__global__ void __launch_bounds__(256) k_l_cdot(const float* __restrict__ a, const float* __restrict__ b, int64_t ld,
                                                int64_t n, double* __restrict__ out) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float re = 0.f, im = 0.f;
  if (k < n) {
    const int64_t o = int64_t(c) * ld + k;
    const float2 x = reinterpret_cast<const float2*>(a)[o], y = reinterpret_cast<const float2*>(b)[o];
    re = x.x * y.x + x.y * y.y;
    im = x.x * y.y - x.y * y.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out + 2 * c, double(re));
    atomicAdd(out + 2 * c + 1, double(im));
  }
}

// out = a + (br + i bi) b over complex64 columns of n entries (stride ld)
__global__ void k_l_axpy(const float* __restrict__ a, const float* __restrict__ b, int64_t ld, int64_t n, float br,
                         float bi, float* __restrict__ out) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t o = int64_t(c) * ld + k;
  const float2 x = reinterpret_cast<const float2*>(a)[o], y = reinterpret_cast<const float2*>(b)[o];
  reinterpret_cast<float2*>(out)[o] = make_float2(x.x + br * y.x - bi * y.y, x.y + br * y.y + bi * y.x);
}

// G3 = 2 w (y - t) and loss += sum w |y - t|^2 (network-level loss)
__global__ void __launch_bounds__(256) k_l_loss(const float* __restrict__ Y, const float* __restrict__ T,
                                                const float* __restrict__ w, int64_t ld, int64_t rows,
                                                float* __restrict__ G3, double* __restrict__ loss) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (q < rows) {
    const float wq = w[q];
    for (int o = 0; o < kLO; ++o) {
      const float d = Y[o * ld + q] - T[o * ld + q];
      G3[o * ld + q] = 2.f * wq * d;
      l += wq * d * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, double(l));
}

__global__ void k_l_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                         float* __restrict__ v, int n, float lr_t, float b1, float b2, float eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  th[k] -= lr_t * mk / (sqrtf(vk) + eps);
}

// D and N complex indices of global dof row g
struct DofIdx {
  int64_t d, n;
};
__device__ __forceinline__ DofIdx l_dof(int64_t g, const int32_t* row_blk, const int32_t* blk_N,
                                        const int64_t* blk_dof_off, const int64_t* blk_row_off) {
  const int i = row_blk[g];
  const int64_t m = g - blk_row_off[i], off = blk_dof_off[i];
  return {off + m, off + blk_N[i] + m};
}

// out = C r for row g of column c (coef kLO x n_rows, src r and pr = P r)
__global__ void __launch_bounds__(256) k_l_stencil(const float* __restrict__ coef, const float* __restrict__ r,
                                                   int64_t ldr, const float* __restrict__ pr, int64_t ldp,
                                                   int64_t n_rows, const int32_t* __restrict__ nbr,
                                                   const int32_t* __restrict__ row_blk,
                                                   const int32_t* __restrict__ blk_N,
                                                   const int64_t* __restrict__ blk_dof_off,
                                                   const int64_t* __restrict__ blk_row_off, float* __restrict__ out,
                                                   int64_t ldo) {
  const int c = blockIdx.y;
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= n_rows) return;
  const float2* rc = reinterpret_cast<const float2*>(r) + int64_t(c) * ldr;
  const float2* pc = reinterpret_cast<const float2*>(pr) + int64_t(c) * ldp;
  float2 zD = make_float2(0.f, 0.f), zN = zD;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const DofIdx id = l_dof(q == 0 ? g : nbr[4 * g + q - 1], row_blk, blk_N, blk_dof_off, blk_row_off);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float2 sD = s == 0 ? rc[id.d] : pc[id.d], sN = s == 0 ? rc[id.n] : pc[id.n];
      const float* a = coef + int64_t((q * 2 + s) * 8) * n_rows + g;  // DD, DN, ND, NN (re, im)
      const float ar0 = a[0], ai0 = a[n_rows], ar1 = a[2 * n_rows], ai1 = a[3 * n_rows];
      const float ar2 = a[4 * n_rows], ai2 = a[5 * n_rows], ar3 = a[6 * n_rows], ai3 = a[7 * n_rows];
      zD.x += ar0 * sD.x - ai0 * sD.y + ar1 * sN.x - ai1 * sN.y;
      zD.y += ar0 * sD.y + ai0 * sD.x + ar1 * sN.y + ai1 * sN.x;
      zN.x += ar2 * sD.x - ai2 * sD.y + ar3 * sN.x - ai3 * sN.y;
      zN.y += ar2 * sD.y + ai2 * sD.x + ar3 * sN.y + ai3 * sN.x;
    }
  }
  const DofIdx me = l_dof(g, row_blk, blk_N, blk_dof_off, blk_row_off);
  float2* oc = reinterpret_cast<float2*>(out) + int64_t(c) * ldo;
  oc[me.d] = zD;
  oc[me.n] = zN;
}

// G3 += dL/da of the stencil coefficients of row g, summed over ncols
// columns: (re, im) of g conj(source) per coefficient, with g = dL/dRe z +
// i dL/dIm z = (sr + i si) w_c for the output z = C(r_c, pr_c)
__global__ void __launch_bounds__(128) k_l_coefgrad(const float* __restrict__ w, const float* __restrict__ r,
                                                    const float* __restrict__ pr, int64_t ld, int ncols, float sr,
                                                    float si, int64_t n_rows, const int32_t* __restrict__ nbr,
                                                    const int32_t* __restrict__ row_blk,
                                                    const int32_t* __restrict__ blk_N,
                                                    const int64_t* __restrict__ blk_dof_off,
                                                    const int64_t* __restrict__ blk_row_off,
                                                    float* __restrict__ G3) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= n_rows) return;
  DofIdx id[5];
#pragma unroll
  for (int q = 0; q < 5; ++q)
    id[q] = l_dof(q == 0 ? g : nbr[4 * g + q - 1], row_blk, blk_N, blk_dof_off, blk_row_off);
  float acc[kLO];
#pragma unroll
  for (int o = 0; o < kLO; ++o) acc[o] = 0.f;
  for (int c = 0; c < ncols; ++c) {
    const float2* wc = reinterpret_cast<const float2*>(w) + int64_t(c) * ld;
    const float2* rc = reinterpret_cast<const float2*>(r) + int64_t(c) * ld;
    const float2* pc = reinterpret_cast<const float2*>(pr) + int64_t(c) * ld;
    const float2 wD = wc[id[0].d], wN = wc[id[0].n];
    const float2 gD = make_float2(sr * wD.x - si * wD.y, sr * wD.y + si * wD.x);
    const float2 gN = make_float2(sr * wN.x - si * wN.y, sr * wN.y + si * wN.x);
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const float2 sD = s == 0 ? rc[id[q].d] : pc[id[q].d], sN = s == 0 ? rc[id[q].n] : pc[id[q].n];
        float* a = acc + (q * 2 + s) * 8;
        // g conj(x) = (g.x x.x + g.y x.y) + i (g.y x.x - g.x x.y)
        a[0] += gD.x * sD.x + gD.y * sD.y;  // DD
        a[1] += gD.y * sD.x - gD.x * sD.y;
        a[2] += gD.x * sN.x + gD.y * sN.y;  // DN
        a[3] += gD.y * sN.x - gD.x * sN.y;
        a[4] += gN.x * sD.x + gN.y * sD.y;  // ND
        a[5] += gN.y * sD.x - gN.x * sD.y;
        a[6] += gN.x * sN.x + gN.y * sN.y;  // NN
        a[7] += gN.y * sN.x - gN.x * sN.y;
      }
  }
#pragma unroll
  for (int o = 0; o < kLO; ++o) G3[o * n_rows + g] += acc[o];
}

// Adjoint of the stencil for row q of column c: out_r = C_r^H w, out_p =
// C_P^H w.  Row m's stencil contains q exactly when q's contains m (the
// neighbour relation is symmetric), at slot 0 for m = q and slot[4 q + k]
// for m = nbr[4 q + k]; the 2 x 2 coupling enters conjugate-transposed.
__global__ void __launch_bounds__(256) k_l_stencil_adj(const float* __restrict__ coef, const float* __restrict__ w,
                                                       int64_t ldw, int64_t n_rows, const int32_t* __restrict__ nbr,
                                                       const int32_t* __restrict__ slot,
                                                       const int32_t* __restrict__ row_blk,
                                                       const int32_t* __restrict__ blk_N,
                                                       const int64_t* __restrict__ blk_dof_off,
                                                       const int64_t* __restrict__ blk_row_off,
                                                       float* __restrict__ out_r, float* __restrict__ out_p,
                                                       int64_t ldo) {
  const int c = blockIdx.y;
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n_rows) return;
  const float2* wc = reinterpret_cast<const float2*>(w) + int64_t(c) * ldw;
  float2 oD[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, oN[2] = {oD[0], oD[0]};
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int64_t mrow = t == 0 ? q : nbr[4 * q + t - 1];
    const int sl = t == 0 ? 0 : slot[4 * q + t - 1];
    const DofIdx id = l_dof(mrow, row_blk, blk_N, blk_dof_off, blk_row_off);
    const float2 wD = wc[id.d], wN = wc[id.n];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float* a = coef + int64_t((sl * 2 + s) * 8) * n_rows + mrow;
      const float ar0 = a[0], ai0 = a[n_rows], ar1 = a[2 * n_rows], ai1 = a[3 * n_rows];
      const float ar2 = a[4 * n_rows], ai2 = a[5 * n_rows], ar3 = a[6 * n_rows], ai3 = a[7 * n_rows];
      // conj(a) w = (ar w.x + ai w.y) + i (ar w.y - ai w.x)
      oD[s].x += ar0 * wD.x + ai0 * wD.y + ar2 * wN.x + ai2 * wN.y;  // conj(DD) w_D + conj(ND) w_N
      oD[s].y += ar0 * wD.y - ai0 * wD.x + ar2 * wN.y - ai2 * wN.x;
      oN[s].x += ar1 * wD.x + ai1 * wD.y + ar3 * wN.x + ai3 * wN.y;  // conj(DN) w_D + conj(NN) w_N
      oN[s].y += ar1 * wD.y - ai1 * wD.x + ar3 * wN.y - ai3 * wN.x;
    }
  }
  const DofIdx me = l_dof(q, row_blk, blk_N, blk_dof_off, blk_row_off);
  float2* orc = reinterpret_cast<float2*>(out_r) + int64_t(c) * ldo;
  float2* opc = reinterpret_cast<float2*>(out_p) + int64_t(c) * ldo;
  orc[me.d] = oD[0];
  orc[me.n] = oN[0];
  opc[me.d] = oD[1];
  opc[me.n] = oN[1];
}

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) of the
// state `x` + golden gamma: a counter-based generator, draw k = mix(seed + k)
__device__ __forceinline__ uint64_t l_splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// complex Rademacher entries (+-1 +- i) / sqrt(2): entry k of column c is
// draw (ctr0 + c) n + k of the generator seeded with `seed`
__global__ void k_l_rademacher(float* __restrict__ z, int64_t n, uint64_t seed, uint64_t ctr0) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint64_t h = l_splitmix64(seed + (ctr0 + uint64_t(c)) * uint64_t(n) + uint64_t(k));
  const float v = 0.70710678f;
  reinterpret_cast<float2*>(z)[int64_t(c) * n + k] = make_float2((h & 1) ? v : -v, (h & 2) ? v : -v);
}

// out^c = f / ss[c] * v^c (0 where ss[c] = 0)
__global__ void k_l_scale_cols(const float* __restrict__ v, int64_t ld, int64_t n, const double* __restrict__ ss,
                               double f, float* __restrict__ out) {
  const int c = blockIdx.y;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float sc = ss[c] > 0 ? float(f / ss[c]) : 0.f;
  const float2 x = reinterpret_cast<const float2*>(v)[int64_t(c) * ld + k];
  reinterpret_cast<float2*>(out)[int64_t(c) * ld + k] = make_float2(sc * x.x, sc * x.y);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static LearnedState& state(mtf_system sys) {
  MTF_REQUIRE(sys->learned != nullptr, MTF_ERR_ARG, "the learned correction has not been initialised");
  return *sys->learned;
}

static void ensure_rows(LearnedState& L, int64_t rows) {
  if (rows <= L.rows_cap) return;
  L.H1.alloc(size_t(kLH) * rows);
  L.H2.alloc(size_t(kLH) * rows);
  L.G2.alloc(size_t(kLH) * rows);
  L.G1.alloc(size_t(kLH) * rows);
  L.Y.alloc(size_t(kLO) * rows);
  L.G3.alloc(size_t(kLO) * rows);
  L.rows_cap = rows;
}

static void ensure_cols(DevBuf<float>& b, int64_t n, int cols) {
  if (b.n < size_t(2 * n) * cols) b.alloc(size_t(2 * n) * cols);
}

int64_t learned_param_count(mtf_system sys) { return sys->learned ? sys->learned->nparam : 0; }

int learned_kind(mtf_system sys) { return state(sys).kind; }

// stencil coefficients in use (kLO x n_rows)
static const float* coef_of(const LearnedState& L) { return L.kind == MTF_LEARNED_TABLE ? L.params.p : L.coef.p; }

// operand helpers for the network products: a feature-major matrix read as
// rows = dofs (A of a forward product), or as rows = features (A or B of a
// weight gradient), and a row-major augmented weight matrix [W | b]
static TgOperand dof_rows(const float* X, int64_t ld, int64_t rows, int feats, bool ones) {
  TgOperand o;
  o.X = X;
  o.sr = 1;
  o.sk = ld;
  o.Rv = rows;
  o.Kv = feats;
  o.ones_k = ones ? feats : -1;
  return o;
}
static TgOperand feat_rows(const float* X, int64_t ld, int feats, int64_t rows, bool ones) {
  TgOperand o;
  o.X = X;
  o.sr = ld;
  o.sk = 1;
  o.Rv = feats;
  o.Kv = rows;
  o.ones_r = ones ? feats : -1;
  return o;
}
static TgOperand weights(const float* W, int outs, int ins_aug) {  // W(c, k) = W[c ins_aug + k]
  TgOperand o;
  o.X = W;
  o.sr = ins_aug;
  o.sk = 1;
  o.Rv = outs;
  o.Kv = ins_aug;
  return o;
}
static TgOperand weights_t(const float* W, int outs, int ins, int ins_aug) {  // W^T(c, k) = W[k ins_aug + c]
  TgOperand o;
  o.X = W;
  o.sr = 1;
  o.sk = ins_aug;
  o.Rv = ins;
  o.Kv = outs;
  return o;
}
static TgOut to_feat(float* D, int64_t ld, int op, const float* mask, unsigned* err) {
  TgOut o;
  o.D = D;
  o.dr = 1;
  o.dc = ld;
  o.op = op;
  o.mask = mask;
  o.mr = 1;
  o.mc = ld;
  o.err = err;
  return o;
}
static TgOut to_weights(float* D, int ins_aug, unsigned* err) {
  TgOut o;
  o.D = D;
  o.dr = ins_aug;
  o.dc = 1;
  o.err = err;
  return o;
}

// forward pass: H1 = relu(W1 [x; 1]), H2 = relu(W2 [H1; 1]), Y = W3 [H2; 1]
// (feature-major, leading dimension ld; H1, H2 kept in L for the backward)
static void forward(mtf_system sys, LearnedState& L, const float* X, int64_t ld, int64_t rows, float* Y,
                    cudaStream_t s) {
  if (!L.gemm) L.gemm = tg_create();
  stream_prepare(sys, s);
  unsigned* err = sys->d_mv_ctl.p + 2;
  const float* W1 = L.params.p;
  const float* W2 = W1 + kLW1;
  const float* W3 = W2 + kLW2;
  tc_gemm(*L.gemm, dof_rows(X, ld, rows, kLF, true), weights(W1, kLH, kLF + 1), rows, kLH, kLF + 1,
          to_feat(L.H1.p, ld, 1, nullptr, err), s);
  tc_gemm(*L.gemm, dof_rows(L.H1.p, ld, rows, kLH, true), weights(W2, kLH, kLH + 1), rows, kLH, kLH + 1,
          to_feat(L.H2.p, ld, 1, nullptr, err), s);
  tc_gemm(*L.gemm, dof_rows(L.H2.p, ld, rows, kLH, true), weights(W3, kLO, kLH + 1), rows, kLO, kLH + 1,
          to_feat(Y, ld, 0, nullptr, err), s);
  check_matvec_stream(sys, s);
}

// network parameter gradient (into L.grad) from dL/dY in L.G3, after a
// forward pass (H1, H2 in L; all with leading dimension rows):
//   G2 = (W3^T G3) masked by H2 > 0, G1 = (W2^T G2) masked by H1 > 0,
//   dW3 = G3 [H2; 1]^T, dW2 = G2 [H1; 1]^T, dW1 = G1 [x; 1]^T
static void backward_from_g3(mtf_system sys, LearnedState& L, const float* X, int64_t rows, cudaStream_t s) {
  const int64_t ld = rows;
  unsigned* err = sys->d_mv_ctl.p + 2;
  const float* W2 = L.params.p + kLW1;
  const float* W3 = W2 + kLW2;
  tc_gemm(*L.gemm, dof_rows(L.G3.p, ld, rows, kLO, false), weights_t(W3, kLO, kLH, kLH + 1), rows, kLH, kLO,
          to_feat(L.G2.p, ld, 2, L.H2.p, err), s);
  tc_gemm(*L.gemm, dof_rows(L.G2.p, ld, rows, kLH, false), weights_t(W2, kLH, kLH, kLH + 1), rows, kLH, kLH,
          to_feat(L.G1.p, ld, 2, L.H1.p, err), s);
  float* dW1 = L.grad.p;
  float* dW2 = dW1 + kLW1;
  float* dW3 = dW2 + kLW2;
  tc_gemm(*L.gemm, feat_rows(L.G3.p, ld, kLO, rows, false), feat_rows(L.H2.p, ld, kLH, rows, true), kLO, kLH + 1,
          rows, to_weights(dW3, kLH + 1, err), s);
  tc_gemm(*L.gemm, feat_rows(L.G2.p, ld, kLH, rows, false), feat_rows(L.H1.p, ld, kLH, rows, true), kLH, kLH + 1,
          rows, to_weights(dW2, kLH + 1, err), s);
  tc_gemm(*L.gemm, feat_rows(L.G1.p, ld, kLH, rows, false), feat_rows(X, ld, kLF, rows, true), kLH, kLF + 1, rows,
          to_weights(dW1, kLF + 1, err), s);
  check_matvec_stream(sys, s);
}

// network: coefficients of the current parameters for every dof
static void refresh_coef(mtf_system sys, cudaStream_t s) {
  LearnedState& L = state(sys);
  if (L.kind != MTF_LEARNED_NETWORK) return;
  const int64_t rows = sys->mesh->n_rows;
  forward(sys, L, L.X.p, rows, rows, L.coef.p, s);
}

void learned_init(mtf_system sys, int kind, uint64_t seed, cudaStream_t s) {
  MTF_REQUIRE(kind == MTF_LEARNED_TABLE || kind == MTF_LEARNED_NETWORK, MTF_ERR_ARG, "unknown learned kind");
  mtf_mesh m = sys->mesh;
  if (!sys->learned) sys->learned = new LearnedState();
  LearnedState& L = *sys->learned;
  L.kind = kind;
  const int64_t nr = m->n_rows;
  // neighbour table (the other edges of the two triangles of every dof) and
  // the triangles of every dof
  std::vector<std::vector<int32_t>> nb(static_cast<size_t>(nr)), tr(static_cast<size_t>(nr));
  for (int i = 0; i < m->nd; ++i) {
    const auto& B = m->blk[i];
    for (int64_t q = B.bt_off; q < B.bt_off + B.T; ++q)
      for (int a = 0; a < 3; ++a) {
        const size_t g = size_t(B.row_off + m->bt_dof[3 * q + a]);
        tr[g].push_back(int32_t(q));
        for (int b = 0; b < 3; ++b)
          if (a != b) {
            const int32_t o = int32_t(B.row_off + m->bt_dof[3 * q + b]);
            if (std::find(nb[g].begin(), nb[g].end(), o) == nb[g].end()) nb[g].push_back(o);
          }
      }
  }
  std::vector<int32_t> tab(static_cast<size_t>(4 * nr)), slot(static_cast<size_t>(4 * nr));
  std::vector<float> X(static_cast<size_t>(kLF * nr));
  auto normal = [&](int64_t q, double* nv) {
    const double* v = &m->bt_v[size_t(9 * q)];
    const double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
    nv[0] = e1[1] * e2[2] - e1[2] * e2[1];
    nv[1] = e1[2] * e2[0] - e1[0] * e2[2];
    nv[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double l = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]) * double(m->bt_swap[size_t(q)]);
    for (int c = 0; c < 3; ++c) nv[c] /= l;
  };
  auto other = [&](int64_t q, int i) {
    const int32_t t = m->bt_tri[size_t(q)];
    return m->L[2 * t] == i ? m->L[2 * t + 1] : m->L[2 * t];
  };
  for (int64_t g = 0; g < nr; ++g) {
    auto& v = nb[size_t(g)];
    MTF_REQUIRE(v.size() == 4 && tr[size_t(g)].size() == 2, MTF_ERR_MESH, "an RWG dof without exactly two triangles");
    std::sort(v.begin(), v.end());
    for (int q = 0; q < 4; ++q) tab[size_t(4 * g + q)] = v[q];
  }
  for (int64_t g = 0; g < nr; ++g)
    for (int q = 0; q < 4; ++q) {
      const auto& w = nb[size_t(tab[size_t(4 * g + q)])];
      const auto it = std::find(w.begin(), w.end(), int32_t(g));
      MTF_REQUIRE(it != w.end(), MTF_ERR_MESH, "asymmetric RWG neighbour relation");
      slot[size_t(4 * g + q)] = int32_t(1 + (it - w.begin()));
    }
  for (int i = 0; i < m->nd; ++i) {
    const auto& B = m->blk[i];
    const double k = sys->k_re[i];
    for (int r = 0; r < B.N; ++r) {
      const int64_t g = B.row_off + r;
      const auto& v = nb[size_t(g)];
      const auto& t = tr[size_t(g)];
      double n0[3], n1[3];
      normal(t[0], n0);
      normal(t[1], n1);
      float* xg = &X[size_t(g)];
      xg[0] = float(k * m->edge_len[size_t(g)]);
      xg[1 * nr] = float(sys->rho_re[i]);
      xg[2 * nr] = i == 0 ? 1.f : 0.f;
      for (int q = 0; q < 4; ++q) xg[(3 + q) * nr] = float(k * m->edge_len[size_t(v[q])]);
      xg[7 * nr] = float(k * k * (m->bt_area[size_t(t[0])] + m->bt_area[size_t(t[1])]));
      xg[8 * nr] = float(n0[0] * n1[0] + n0[1] * n1[1] + n0[2] * n1[2]);
      xg[9 * nr] = other(t[0], i) != other(t[1], i) ? 1.f : 0.f;
    }
  }
  L.nbr.upload(tab, s);
  L.slot.upload(slot, s);
  L.X.alloc(X.size());
  MTF_CUDA(cudaMemcpyAsync(L.X.p, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  std::vector<float> th;
  if (kind == MTF_LEARNED_TABLE) {
    L.nparam = int64_t(kLO) * nr;
    th.assign(size_t(L.nparam), 0.f);
  } else {
    // He-uniform hidden layers, zero output layer (an untrained network adds nothing)
    L.nparam = kLNetParams;
    th.assign(size_t(L.nparam), 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int rows, int cols) {
      const float bound = std::sqrt(6.f / float(cols - 1));
      std::uniform_real_distribution<float> U(-bound, bound);
      for (int rr = 0; rr < rows; ++rr)
        for (int cc = 0; cc < cols; ++cc) th[size_t(off + rr * cols + cc)] = cc == cols - 1 ? 0.f : U(rng);
    };
    fill(0, kLH, kLF + 1);
    fill(kLW1, kLH, kLH + 1);
    L.coef.alloc(size_t(kLO) * nr);
  }
  L.params.alloc(th.size());
  L.grad.alloc(th.size());
  L.am.alloc(th.size());
  L.av.alloc(th.size());
  MTF_CUDA(cudaMemcpyAsync(L.params.p, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemsetAsync(L.am.p, 0, th.size() * sizeof(float), s));
  MTF_CUDA(cudaMemsetAsync(L.av.p, 0, th.size() * sizeof(float), s));
  L.adam_t = 0;
  L.draws = 0;
  L.acc.alloc(256);
  ensure_rows(L, nr);
  refresh_coef(sys, s);
  MTF_CUDA(cudaStreamSynchronize(s));  // host tables go out of scope
}

void learned_set_params(mtf_system sys, const float* host, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_CUDA(cudaMemcpyAsync(L.params.p, host, size_t(L.nparam) * sizeof(float), cudaMemcpyHostToDevice, s));
  refresh_coef(sys, s);
  MTF_CUDA(cudaStreamSynchronize(s));
}

void learned_get_params(mtf_system sys, float* host, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_CUDA(cudaMemcpyAsync(host, L.params.p, size_t(L.nparam) * sizeof(float), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
}

void learned_features(mtf_system sys, float* X, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_CUDA(cudaMemcpyAsync(X, L.X.p, L.X.n * sizeof(float), cudaMemcpyDeviceToDevice, s));
}

static void sumsq(const float* v, int64_t ld, int64_t n, int ncols, double* out, cudaStream_t s) {
  MTF_CUDA(cudaMemsetAsync(out, 0, size_t(ncols) * sizeof(double), s));
  MTF_LAUNCH(KID_MLP, s, k_l_sumsq<<<dim3(nbk(n, 256), unsigned(ncols)), 256, 0, s>>>(v, ld, n, out));
}

void learned_loss_grad(mtf_system sys, const float* X, const float* T, const float* w, int64_t rows, float* grad_out,
                       double* loss_host, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_REQUIRE(L.kind == MTF_LEARNED_NETWORK, MTF_ERR_ARG, "the network loss needs the network parametrisation");
  MTF_REQUIRE(rows >= 1, MTF_ERR_ARG, "rows must be >= 1");
  ensure_rows(L, rows);
  forward(sys, L, X, rows, rows, L.Y.p, s);
  double* loss_dev = L.acc.p + 255;
  MTF_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(double), s));
  MTF_LAUNCH(KID_MLP, s, k_l_loss<<<nbk(rows, 256), 256, 0, s>>>(L.Y.p, T, w, rows, rows, L.G3.p, loss_dev));
  backward_from_g3(sys, L, X, rows, s);
  MTF_CUDA(cudaMemcpyAsync(grad_out, L.grad.p, kLNetParams * sizeof(float), cudaMemcpyDeviceToDevice, s));
  double l = 0;
  MTF_CUDA(cudaMemcpyAsync(&l, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = l;
}

// C r for r (stride ldr) and pr = P r (stride ldp) into out (stride ldo)
static void stencil(mtf_system sys, const float* r, int64_t ldr, const float* pr, int64_t ldp, int nrhs, float* out,
                    int64_t ldo, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  LearnedState& L = state(sys);
  MTF_LAUNCH(KID_MLP, s, k_l_stencil<<<dim3(nbk(m->n_rows, 256), unsigned(nrhs)), 256, 0, s>>>(
      coef_of(L), r, ldr, pr, ldp, m->n_rows, L.nbr.p, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p,
      m->d_blk_row_off.p, out, ldo));
}

// out_r = C_r^H w, out_p = C_P^H w (all columns of stride n_total)
void learned_stencil_adjoint(mtf_system sys, const float* w, float* out_r, float* out_p, int nrhs, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  LearnedState& L = state(sys);
  const int64_t n = m->n_total;
  MTF_LAUNCH(KID_MLP, s, k_l_stencil_adj<<<dim3(nbk(m->n_rows, 256), unsigned(nrhs)), 256, 0, s>>>(
      coef_of(L), w, n, m->n_rows, L.nbr.p, L.slot.p, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p,
      m->d_blk_row_off.p, out_r, out_p, n));
}

// z (= P r on entry) += C r for nrhs columns (column strides ldr, ldz)
void learned_apply_inplace(mtf_system sys, const float* r, int64_t ldr, float* z, int64_t ldz, int nrhs,
                           cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  LearnedState& L = state(sys);
  const int64_t n = m->n_total;
  ensure_cols(L.CA, ldz, nrhs);
  stencil(sys, r, ldr, z, ldz, nrhs, L.CA.p, ldz, s);
  MTF_LAUNCH(KID_MLP, s, k_l_axpy<<<dim3(nbk(n, 256), unsigned(nrhs)), 256, 0, s>>>(z, L.CA.p, ldz, n, 1.f, 0.f, z));
}

// Power loss on the pb columns of Z (stride n_total) and its gradient with
// respect to the stencil coefficients (into L.G3; network: also L.grad).
// Returns the loss.
static double power_grad(mtf_system sys, const float* Z, int pb, double c0r, double c0i, int K, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  LearnedState& L = state(sys);
  const int64_t n = m->n_total, nr = m->n_rows;
  const size_t col = size_t(2 * n);
  ensure_cols(L.E, n, (K + 1) * pb);
  ensure_cols(L.PE, n, K * pb);
  for (DevBuf<float>* b : {&L.T, &L.MT, &L.A, &L.B, &L.CRH, &L.CPH, &L.U}) ensure_cols(*b, n, pb);
  const dim3 gv{nbk(n, 256), unsigned(pb)};
  const double cn = c0r * c0r + c0i * c0i;
  MTF_REQUIRE(cn > 0, MTF_ERR_ARG, "c0 must not be zero");
  // ic = 1 / c0; forward steps use -ic, backward steps -conj(ic)
  const float icr = float(c0r / cn), ici = float(-c0i / cn);
  if (L.kind == MTF_LEARNED_NETWORK) forward(sys, L, L.X.p, nr, nr, L.coef.p, s);
  MTF_CUDA(cudaMemcpyAsync(L.E.p, Z, col * pb * sizeof(float), cudaMemcpyDeviceToDevice, s));
  for (int j = 0; j < K; ++j) {
    float* Ej = L.E.p + col * pb * j;
    float* PEj = L.PE.p + col * pb * j;
    launch_osrc_apply_f32(sys, Ej, n, PEj, n, pb, s);
    stencil(sys, Ej, n, PEj, n, pb, L.T.p, n, s);
    MTF_LAUNCH(KID_MLP, s, k_l_axpy<<<gv, 256, 0, s>>>(PEj, L.T.p, n, n, 1.f, 0.f, L.T.p));
    launch_matvec_f32(sys, L.T.p, n, L.MT.p, n, pb, s);
    MTF_LAUNCH(KID_MLP, s, k_l_axpy<<<gv, 256, 0, s>>>(Ej, L.MT.p, n, n, -icr, -ici, Ej + col * pb));
  }
  double* ssz = L.acc.p;
  double* sse = L.acc.p + 64;
  const float* EK = L.E.p + col * pb * K;
  sumsq(Z, n, n, pb, ssz, s);
  sumsq(EK, n, n, pb, sse, s);
  MTF_LAUNCH(KID_MLP, s, k_l_scale_cols<<<gv, 256, 0, s>>>(EK, n, n, ssz, 2.0 / pb, L.A.p));
  MTF_CUDA(cudaMemsetAsync(L.G3.p, 0, size_t(kLO) * nr * sizeof(float), s));
  for (int j = K - 1; j >= 0; --j) {
    const float* Ej = L.E.p + col * pb * j;
    const float* PEj = L.PE.p + col * pb * j;
    launch_matvec_adj_f32(sys, L.A.p, n, L.B.p, n, pb, s);
    MTF_LAUNCH(KID_MLP, s, k_l_coefgrad<<<nbk(nr, 128), 128, 0, s>>>(
        L.B.p, Ej, PEj, n, pb, -icr, ici, nr, L.nbr.p, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p,
        m->d_blk_row_off.p, L.G3.p));
    if (j == 0) break;
    learned_stencil_adjoint(sys, L.B.p, L.CRH.p, L.CPH.p, pb, s);
    MTF_LAUNCH(KID_MLP, s, k_l_axpy<<<gv, 256, 0, s>>>(L.B.p, L.CPH.p, n, n, 1.f, 0.f, L.CPH.p));
    launch_osrc_apply_adj_f32(sys, L.CPH.p, n, L.U.p, n, pb, s);
    MTF_LAUNCH(KID_MLP, s, k_l_axpy<<<gv, 256, 0, s>>>(L.U.p, L.CRH.p, n, n, 1.f, 0.f, L.U.p));
    MTF_LAUNCH(KID_MLP, s, k_l_axpy<<<gv, 256, 0, s>>>(L.A.p, L.U.p, n, n, -icr, ici, L.A.p));
  }
  if (L.kind == MTF_LEARNED_NETWORK) backward_from_g3(sys, L, L.X.p, nr, s);
  std::vector<double> h(static_cast<size_t>(128), 0.0);
  MTF_CUDA(cudaMemcpyAsync(h.data(), L.acc.p, 128 * sizeof(double), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  double loss = 0;
  for (int c = 0; c < pb; ++c)
    if (h[size_t(c)] > 0) loss += h[size_t(64 + c)] / h[size_t(c)];
  return loss / pb;
}

static const float* grad_of(const LearnedState& L) { return L.kind == MTF_LEARNED_TABLE ? L.G3.p : L.grad.p; }

void learned_power_grad(mtf_system sys, const float* Z, int pb, double c0r, double c0i, int K, float* grad_out,
                        double* loss_host, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_REQUIRE(sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG, "training needs a mixed-precision system");
  MTF_REQUIRE(pb >= 1 && pb <= kLMaxBatch && K >= 1 && K <= kLMaxK, MTF_ERR_ARG, "1 <= columns <= 32, 1 <= K <= 16");
  const double l = power_grad(sys, Z, pb, c0r, c0i, K, s);
  MTF_CUDA(cudaMemcpyAsync(grad_out, grad_of(L), size_t(L.nparam) * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  check_matvec_stream(sys, s);
  if (loss_host) *loss_host = l;
}

// next `cols` random training vectors into L.Zb
static void draw(mtf_system sys, uint64_t seed, int cols, cudaStream_t s) {
  LearnedState& L = state(sys);
  const int64_t n = sys->mesh->n_total;
  ensure_cols(L.Zb, n, cols);
  MTF_LAUNCH(KID_MLP, s, k_l_rademacher<<<dim3(nbk(n, 256), unsigned(cols)), 256, 0, s>>>(L.Zb.p, n, seed, L.draws));
  L.draws += uint64_t(cols);
}

// c0 = mean over 64 random vectors of <z, M P z> / <z, z>, P plain block-OSRC
static void estimate_centre(mtf_system sys, uint64_t seed, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  LearnedState& L = state(sys);
  const int64_t n = m->n_total;
  const int pb = kLMaxBatch;
  ensure_cols(L.T, n, pb);
  ensure_cols(L.MT, n, pb);
  double* dots = L.acc.p + 64;
  double* ssz = L.acc.p;
  std::vector<double> hd(static_cast<size_t>(2 * pb)), hn(static_cast<size_t>(pb));
  double cr = 0, ci = 0;
  int used = 0;
  for (int rep = 0; rep < 2; ++rep) {
    draw(sys, seed, pb, s);
    launch_osrc_apply_f32(sys, L.Zb.p, n, L.T.p, n, pb, s);
    launch_matvec_f32(sys, L.T.p, n, L.MT.p, n, pb, s);
    MTF_CUDA(cudaMemsetAsync(dots, 0, size_t(2 * pb) * sizeof(double), s));
    MTF_LAUNCH(KID_MLP, s, k_l_cdot<<<dim3(nbk(n, 256), unsigned(pb)), 256, 0, s>>>(L.Zb.p, L.MT.p, n, n, dots));
    sumsq(L.Zb.p, n, n, pb, ssz, s);
    MTF_CUDA(cudaMemcpyAsync(hd.data(), dots, size_t(2 * pb) * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaMemcpyAsync(hn.data(), ssz, size_t(pb) * sizeof(double), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    for (int c = 0; c < pb; ++c) {
      cr += hd[size_t(2 * c)] / hn[size_t(c)];
      ci += hd[size_t(2 * c + 1)] / hn[size_t(c)];
      ++used;
    }
  }
  check_matvec_stream(sys, s);
  L.center_re = cr / used;
  L.center_im = ci / used;
  L.centred = true;
}

double learned_centre(mtf_system sys, double* im, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_REQUIRE(sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG, "the centre needs a mixed-precision system");
  if (!L.centred) estimate_centre(sys, 0x5eed5eedull, s);
  if (im) *im = L.center_im;
  return L.center_re;
}

void learned_train(mtf_system sys, int steps, double lr, int batch, int K, uint64_t seed, double* loss_first,
                   double* loss_last, cudaStream_t s) {
  LearnedState& L = state(sys);
  MTF_REQUIRE(sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG, "training needs a mixed-precision system");
  MTF_REQUIRE(steps >= 0 && batch >= 1 && batch <= kLMaxBatch && K >= 1 && K <= kLMaxK && lr > 0, MTF_ERR_ARG,
              "steps >= 0, 1 <= batch <= 32, 1 <= K <= 16, lr > 0");
  double c0i = 0;
  const double c0r = learned_centre(sys, &c0i, s);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double first = 0, last = 0;
  for (int st = 0; st < steps; ++st) {
    draw(sys, seed, batch, s);
    const double l = power_grad(sys, L.Zb.p, batch, c0r, c0i, K, s);
    if (st == 0) first = l;
    last = l;
    ++L.adam_t;
    const double lr_t = lr * std::sqrt(1.0 - std::pow(double(b2), double(L.adam_t))) /
                        (1.0 - std::pow(double(b1), double(L.adam_t)));
    MTF_LAUNCH(KID_MLP, s, k_l_adam<<<nbk(L.nparam, 256), 256, 0, s>>>(
        L.params.p, grad_of(L), L.am.p, L.av.p, int(L.nparam), float(lr_t), b1, b2, eps));
  }
  refresh_coef(sys, s);
  MTF_CUDA(cudaStreamSynchronize(s));
  check_matvec_stream(sys, s);
  if (loss_first) *loss_first = first;
  if (loss_last) *loss_last = last;
}

}  // namespace mtf
