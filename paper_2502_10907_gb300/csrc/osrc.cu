// Block-OSRC preconditioner of Sec. 4.4 (Eq. 19):
//   A~_i = [[0, rho_i^-1 T~], [-rho_i T~, 0]],  T~ ~ EtM ~ T^-1.
// Discretisation (the paper leaves it to the cited OSRC work): RWG_i splits
// G-orthogonally (G the RWG mass) into irrotational modes, eigenpairs
// D v = lambda G v (lambda > 0, D the div-div matrix, |xi|^2 = lambda), and
// loop modes L phi / sqrt(mu) from the P1 Laplace-Beltrami eigenpairs
// S phi = mu M phi (L phi = RWG coefficients of n x grad phi, |xi|^2 = mu).
// With W the G-orthonormal basis of both and Z = -|xi|^2 / k_eps^2,
//   T~ = W diag(f) W^T,  f = 2k / (k_eps P(Z)) (irrotational),
//                        f = (2 k_eps / k) P(Z) (loops),
// where P is the rotating-branch-cut Pade approximant of sqrt(1 + z) of order
// N_p and angle theta (Milinazzo, Zala & Brooke 1997) and k_eps = k + i eps,
// eps = c k^{1/3} R^{-2/3}, R the radius of the sphere with Gamma_i's area.
// the two factors of the OSRC magnetic-to-electric operator.  The eigenpairs
// depend on the mesh only and are computed once (FP32 dense symmetric-
// definite eigensolver); f depends on k and is recomputed at every assembly,
// together with the dense complex T~ of every block (two FP32 GEMMs,
// W diag(Re f) W^T and W diag(Im f) W^T).  The apply streams T~ once per
// right-hand-side chunk with the bulk-copy row kernel (stream.cuh, ENT = 1),
// HBM-bound like the block matvec: the same bytes as the two real passes
// t = W^T r, z = W (f t), in one launch and without the intermediate t.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>

#include "stream.cuh"
#include "stream_tc.cuh"

// FP16 T~ applies on the tensor cores (stream_tc.cuh); 0 keeps the FMA
// stream of stream.cuh for them
#ifndef MTF_OSRC_TC
#define MTF_OSRC_TC 1
#endif

namespace mtf {

__constant__ double c_os_s[6], c_os_t[6], c_os_w[6];

// dense G and D of every block (FP32, column-major = row-major, symmetric)
__global__ void k_gram_divdiv(const double* __restrict__ bt_v, const double* __restrict__ bt_c,
                              const double* __restrict__ bt_area, const int32_t* __restrict__ bt_dof,
                              const int32_t* __restrict__ bt_blk, const int64_t* __restrict__ blk_mat_off,
                              const int32_t* __restrict__ blk_N, int64_t n_bt, float* __restrict__ G,
                              float* __restrict__ D) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n_bt) return;
  const int i = bt_blk[q];
  const int N = blk_N[i];
  const int64_t base = blk_mat_off[i];
  const double* v = bt_v + 9 * q;
  const double A2 = 2.0 * bt_area[q];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double g = 0.0;
      for (int p = 0; p < 6; ++p) {
        double dot = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double x = v[c] + c_os_s[p] * (v[3 + c] - v[c]) + c_os_t[p] * (v[6 + c] - v[c]);
          dot += (x - v[3 * a + c]) * (x - v[3 * b + c]);
        }
        g += c_os_w[p] * dot;
      }
      const double ca = bt_c[3 * q + a], cb = bt_c[3 * q + b];
      const int64_t e = base + int64_t(bt_dof[3 * q + a]) * N + bt_dof[3 * q + b];
      atomicAdd(G + e, float(A2 * g * ca * cb));
      atomicAdd(D + e, float(0.5 * A2 * (2.0 * ca) * (2.0 * cb)));
    }
}

// dense P1 Laplace-Beltrami stiffness S and mass M of every block
__global__ void k_p1_matrices(const double* __restrict__ bt_v, const double* __restrict__ bt_area,
                              const int32_t* __restrict__ bt_lv, const int32_t* __restrict__ bt_blk,
                              const int64_t* __restrict__ p1_off, const int32_t* __restrict__ p1_n, int64_t n_bt,
                              float* __restrict__ S, float* __restrict__ M) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n_bt) return;
  const int i = bt_blk[q];
  const int nv = p1_n[i];
  const double* P = bt_v + 9 * q;
  const double A = bt_area[q];
  double e1[3], e2[3], n[3];
  for (int c = 0; c < 3; ++c) {
    e1[c] = P[3 + c] - P[c];
    e2[c] = P[6 + c] - P[c];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  double g[3][3];  // grad of barycentric a = n x (P_{a+2} - P_{a+1}) / |n|^2
  for (int a = 0; a < 3; ++a) {
    double t[3];
    for (int c = 0; c < 3; ++c) t[c] = P[3 * ((a + 2) % 3) + c] - P[3 * ((a + 1) % 3) + c];
    g[a][0] = (n[1] * t[2] - n[2] * t[1]) / nn;
    g[a][1] = (n[2] * t[0] - n[0] * t[2]) / nn;
    g[a][2] = (n[0] * t[1] - n[1] * t[0]) / nn;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const int64_t e = p1_off[i] + int64_t(bt_lv[3 * q + a]) * nv + bt_lv[3 * q + b];
      atomicAdd(S + e, float(A * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2])));
      atomicAdd(M + e, float(A * (a == b ? 2.0 : 1.0) / 12.0));
    }
}

// W (column-major, N x N per block): columns j < nirr the irrotational
// eigenvectors V[:, N - nirr + j]; columns nirr + k (k < nv - 1) the loop
// modes L Phi[:, k+1] / sqrt(mu_{k+1}), L[e, lo] = 1/l_e, L[e, hi] = -1/l_e;
// the remaining 2 g columns (harmonic fields of a genus-g boundary) are
// zeroed here and filled by osrc_harmonic.  eig[row_off + j] receives the
// matching |xi|^2 (0 for the harmonic fields).
__global__ void k_build_w(const float* __restrict__ V, const float* __restrict__ lam, const float* __restrict__ Phi,
                          const float* __restrict__ mu, const int32_t* __restrict__ edge_lohi,
                          const double* __restrict__ edge_len, int N, int nirr, int nv, float* __restrict__ W,
                          float* __restrict__ eig) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(N) * N) return;
  const int j = int(t / N), e = int(t % N);  // column j, row e
  float v;
  if (j < nirr) {
    v = V[int64_t(N - nirr + j) * N + e];
    if (e == 0) eig[j] = lam[N - nirr + j];
  } else if (j >= nirr + nv - 1) {
    v = 0.f;
    if (e == 0) eig[j] = 0.f;
  } else {
    const int k = j - nirr + 1;
    const float* ph = Phi + int64_t(k) * nv;
    const float sm = sqrtf(fmaxf(mu[k], 1e-30f));
    v = float((ph[edge_lohi[2 * e]] - ph[edge_lohi[2 * e + 1]]) / (edge_len[e] * sm));
    if (e == 0) eig[j] = mu[k];
  }
  W[t] = v;
}

// W^T row-major padded (ld): row j = column j of W; pad entries are zero
__global__ void k_pad_copy(const float* __restrict__ W, int N, int ld, float* __restrict__ Wt) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(N) * ld) return;
  const int j = int(t / ld), e = int(t % ld);
  Wt[t] = e < N ? W[int64_t(j) * N + e] : 0.0f;
}

// symbol per (block, mode j) with Z = -|xi|^2 / k_eps^2:
//   irrotational (j < nirr): f = 2k / (k_eps P(Z)),  loop: f = (2 k_eps / k) P(Z)
// type2: the modulus of f with the phase of the EtM principal symbols,
//   -i |f| on irrotational modes, +i |f| on loop and harmonic modes
// (block-OSRC Type 2: T~2 = W diag(f2) W^T = i R with R real symmetric)
__global__ void k_osrc_symbol(const float* __restrict__ lam, const int32_t* __restrict__ row_blk, int64_t n_rows,
                              const int64_t* __restrict__ blk_row_off, const int32_t* __restrict__ nirr_blk,
                              const double* __restrict__ kk, const double* __restrict__ keps,
                              const double* __restrict__ pd, int np, int type2, float2* __restrict__ f) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int i = row_blk[r];
  const bool irr = (r - blk_row_off[i]) < nirr_blk[i];
  // complex arithmetic written out: (re, im) pairs
  const double kr = keps[2 * i], ki = keps[2 * i + 1];
  const double k2r = kr * kr - ki * ki, k2i = 2 * kr * ki;          // k_eps^2
  const double k2n = k2r * k2r + k2i * k2i;
  const double l = double(lam[r]);
  const double zr = -l * k2r / k2n, zi = l * k2i / k2n;            // -lambda / k_eps^2
  double Pr = pd[0], Pi = pd[1];
  for (int j = 0; j < np; ++j) {
    const double Ar = pd[2 + 4 * j], Ai = pd[3 + 4 * j], Br = pd[4 + 4 * j], Bi = pd[5 + 4 * j];
    const double nr = Ar * zr - Ai * zi, ni = Ar * zi + Ai * zr;   // A z
    const double dr = 1.0 + Br * zr - Bi * zi, di = Br * zi + Bi * zr;  // 1 + B z
    const double dn = dr * dr + di * di;
    Pr += (nr * dr + ni * di) / dn;
    Pi += (ni * dr - nr * di) / dn;
  }
  const double er = kr * Pr - ki * Pi, ei = kr * Pi + ki * Pr;     // k_eps P
  const double k0 = kk[2 * i];
  double fr, fi;
  if (irr) {
    const double en = er * er + ei * ei;
    fr = 2.0 * k0 * er / en;
    fi = -2.0 * k0 * ei / en;
  } else {
    fr = 2.0 * er / k0;
    fi = 2.0 * ei / k0;
  }
  if (type2) {
    const double a = sqrt(fr * fr + fi * fi);
    fr = 0.0;
    fi = irr ? -a : a;
  }
  f[r] = make_float2(float(fr), float(fi));
}

// z rows of one block row m (one warp per global row): the row's T~ pieces
// added in order, then z_D = rho^-1 (T~ r_N), z_N = -rho (T~ r_D) per
// right-hand side (lane c < NC), in the output precision.
//
// ADJ: the input columns were conjugated (w~ = conj(w)); with T~ symmetric,
// P^H w = conj([-rho T~ w~_N ; rho^-1 T~ w~_D]) is written instead (FP32).
// ENT: entry type of the streamed T~ (1: FP32, 3: FP16 scaled per block, the
// scale folded into rho32).
template <int NC, class ZT, bool ADJ = false, int ENT = 1>
__global__ void __launch_bounds__(256) k_os_combine(const float* __restrict__ part, int pmax,
                                                    const int32_t* __restrict__ row_blk,
                                                    const int32_t* __restrict__ blk_N,
                                                    const int64_t* __restrict__ blk_dof_off,
                                                    const int64_t* __restrict__ blk_row_off,
                                                    const double* __restrict__ rho, const float* __restrict__ rho32,
                                                    ZT* __restrict__ z, int64_t ldz, int c0, int64_t n_rows) {
  MTF_PDL_WAIT();
  MTF_PDL_TRIGGER();
  constexpr int K = StreamK<NC, ENT>::K;
  const int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int i = row_blk[row];
  const int N = blk_N[i];
  const int P = st_pieces<ENT>(N);
  const float tot = st_row_total<K>(part + row * pmax * K, P, lane);
  float a[4];
  const int cl = lane < NC ? lane : 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = __shfl_sync(0xffffffffu, tot, cl * 4 + q);
  if (lane >= NC) return;
  ZT rr, ri, ir, ii;
  if constexpr (sizeof(ZT) == 4) {
    rr = rho32[4 * i];
    ri = rho32[4 * i + 1];
    ir = rho32[4 * i + 2];
    ii = rho32[4 * i + 3];
  } else {
    rr = rho[2 * i];
    ri = rho[2 * i + 1];
    const ZT rn = rr * rr + ri * ri;
    ir = rr / rn;
    ii = -ri / rn;
  }
  const int64_t m = row - blk_row_off[i];
  ZT* zc = z + 2 * (int64_t(c0 + lane) * ldz + blk_dof_off[i]);
  const ZT a0 = a[0], a1 = a[1], a2 = a[2], a3 = a[3];  // T~ r_D, T~ r_N
  if constexpr (ADJ) {
    zc[2 * m] = -(rr * a2 - ri * a3);
    zc[2 * m + 1] = rr * a3 + ri * a2;
    zc[2 * (N + m)] = ir * a0 - ii * a1;
    zc[2 * (N + m) + 1] = -(ir * a1 + ii * a0);
    return;
  }
  zc[2 * m] = ir * a2 - ii * a3;
  zc[2 * m + 1] = ir * a3 + ii * a2;
  zc[2 * (N + m)] = -(rr * a0 - ri * a1);
  zc[2 * (N + m) + 1] = -(rr * a1 + ri * a0);
}

// mx[i] = max over block i's T~ entries of max(|re|, |im|) (non-negative
// floats compare as their bit patterns)
__global__ void k_os_absmax(const float2* __restrict__ T, int64_t n, int blk, unsigned* __restrict__ mx) {
  float a = 0.f;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const float2 v = T[k];
    a = fmaxf(a, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx + blk, __float_as_uint(a));
}

// FP16 copy of one block of T~: rows of ld16 (multiple of 4) entries,
// entries scaled by inv, padding zero
__global__ void k_os_to_half(const float2* __restrict__ T, int N, int ld32, int ld16, float inv,
                             __half2* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= int64_t(N) * ld16) return;
  const int64_t r = k / ld16;
  const int c = int(k - r * ld16);
  const float2 v = c < N ? T[r * ld32 + c] : make_float2(0.f, 0.f);
  out[k] = __floats2half2_rn(v.x * inv, v.y * inv);
}

__global__ void k_to_f32_cols(const double* __restrict__ x, int64_t ldx, int64_t n2, int nrhs, float* __restrict__ out) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n2 * nrhs) return;
  const int64_t c = t / n2, k = t % n2;
  out[t] = float(x[2 * c * ldx + k]);
}

// cuBLAS / cuSOLVER handles: one per device, each used under its device's
// lock (a handle is bound to the device it was created on, and its stream
// setting is shared state), in FP32 pedantic math (no TF32 rounding)
static constexpr int kMaxDev = 64;

// the calling device's cuBLAS handle, bound to stream s, FP32 pedantic math;
// the device's lock is held while the lease lives
struct BlasLease {
  cublasHandle_t h;
  std::unique_lock<std::mutex> lock;
};

static BlasLease blas_lease(cudaStream_t s) {
  static cublasHandle_t h[kMaxDev] = {};
  static std::mutex mu[kMaxDev];
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  MTF_REQUIRE(dev >= 0 && dev < kMaxDev, MTF_ERR_CUDA, "device index out of range");
  BlasLease L{nullptr, std::unique_lock<std::mutex>(mu[dev])};
  if (!h[dev]) {
    MTF_REQUIRE(cublasCreate(&h[dev]) == CUBLAS_STATUS_SUCCESS, MTF_ERR_CUDA, "cublasCreate failed");
    MTF_REQUIRE(cublasSetMathMode(h[dev], CUBLAS_PEDANTIC_MATH) == CUBLAS_STATUS_SUCCESS, MTF_ERR_CUDA,
                "cublasSetMathMode failed");
  }
  MTF_REQUIRE(cublasSetStream(h[dev], s) == CUBLAS_STATUS_SUCCESS, MTF_ERR_CUDA, "cublasSetStream failed");
  L.h = h[dev];
  return L;
}

struct SolverLease {
  cusolverDnHandle_t h;
  std::unique_lock<std::mutex> lock;
};

static SolverLease solver_lease(cudaStream_t s) {
  static cusolverDnHandle_t h[kMaxDev] = {};
  static std::mutex mu[kMaxDev];
  int dev = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  MTF_REQUIRE(dev >= 0 && dev < kMaxDev, MTF_ERR_CUDA, "device index out of range");
  SolverLease L{nullptr, std::unique_lock<std::mutex>(mu[dev])};
  if (!h[dev]) {
    MTF_REQUIRE(cusolverDnCreate(&h[dev]) == CUSOLVER_STATUS_SUCCESS, MTF_ERR_CUDA, "cusolverDnCreate failed");
  }
  MTF_REQUIRE(cusolverDnSetStream(h[dev], s) == CUSOLVER_STATUS_SUCCESS, MTF_ERR_CUDA, "cusolverDnSetStream failed");
  L.h = h[dev];
  return L;
}

// The 2 g harmonic fields of a genus-g boundary (the part of the kernel of
// the div-div pencil that is G-orthogonal to the loop modes): with K the
// first m = N - nirr (G-orthonormal) eigenvectors of (D, G), U the nloop
// loop modes (columns nirr .. nirr + nloop - 1 of W) and R = K - U (U^T G K),
// the m x m matrix R^T G R has eigenvalue 1 on the nh harmonic directions
// and 0 on the loop ones; its top nh eigenvectors Y give the G-orthonormal
// harmonic fields R Y / sqrt(sigma), written into the last nh columns of W.
// G is a copy of the mass matrix (the div-div eigensolver overwrites its
// own).  cuBLAS / cuSOLVER on the stream, FP32 like the rest of the setup.
static void osrc_harmonic(int N, int nirr, int nloop, int nh, const float* K, const float* G, float* W,
                          cusolverDnHandle_t sh, cudaStream_t s) {
  const int m = N - nirr;
  BlasLease bl = blas_lease(s);
  cublasHandle_t bh = bl.h;
  DevBuf<float> GK, X, R, Q, w;
  GK.alloc(size_t(N) * m);
  X.alloc(size_t(std::max(nloop, 1)) * m);
  R.alloc(size_t(N) * m);
  Q.alloc(size_t(m) * m);
  w.alloc(size_t(m));
  const float one = 1.f, zero = 0.f, mone = -1.f;
  const float* U = W + size_t(nirr) * N;
  auto gemm = [&](cublasOperation_t ta, int rows, int cols, int inner, float alpha, const float* Ap, int lda,
                  const float* Bp, int ldb, float beta, float* Cp, int ldc) {
    MTF_REQUIRE(cublasSgemm(bh, ta, CUBLAS_OP_N, rows, cols, inner, &alpha, Ap, lda, Bp, ldb, &beta, Cp, ldc) ==
                    CUBLAS_STATUS_SUCCESS,
                MTF_ERR_CUDA, "cublasSgemm failed (harmonic fields)");
  };
  gemm(CUBLAS_OP_N, N, m, N, one, G, N, K, N, zero, GK.p, N);  // G K
  MTF_CUDA(cudaMemcpyAsync(R.p, K, size_t(N) * m * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (nloop > 0) {
    gemm(CUBLAS_OP_T, nloop, m, N, one, U, N, GK.p, N, zero, X.p, nloop);  // U^T G K
    gemm(CUBLAS_OP_N, N, m, nloop, mone, U, N, X.p, nloop, one, R.p, N);   // R = K - U X
  }
  gemm(CUBLAS_OP_N, N, m, N, one, G, N, R.p, N, zero, GK.p, N);       // G R
  gemm(CUBLAS_OP_T, m, m, N, one, R.p, N, GK.p, N, zero, Q.p, m);     // R^T G R
  int lwork = 0;
  MTF_REQUIRE(cusolverDnSsyevd_bufferSize(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, Q.p, m, w.p,
                                          &lwork) == CUSOLVER_STATUS_SUCCESS,
              MTF_ERR_CUDA, "cusolverDnSsyevd_bufferSize failed");
  DevBuf<float> work;
  work.alloc(size_t(std::max(lwork, 1)));
  DevBuf<int> info;
  info.alloc(1);
  MTF_REQUIRE(cusolverDnSsyevd(sh, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, Q.p, m, w.p, work.p, lwork,
                               info.p) == CUSOLVER_STATUS_SUCCESS,
              MTF_ERR_CUDA, "cusolverDnSsyevd failed");
  std::vector<float> wh(static_cast<size_t>(m));
  int hinfo = 0;
  MTF_CUDA(cudaMemcpyAsync(wh.data(), w.p, size_t(m) * sizeof(float), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  MTF_REQUIRE(hinfo == 0, MTF_ERR_CUDA, "harmonic-field eigensolver failed (info " + std::to_string(hinfo) + ")");
  // nh eigenvalues near 1 above m - nh near 0: the dimension count holds
  MTF_REQUIRE(wh[size_t(m - nh)] > 0.5f && (m == nh || wh[size_t(m - nh - 1)] < 0.5f), MTF_ERR_MESH,
              "harmonic fields of a subdomain boundary not separated from its loop modes");
  float* H = W + size_t(nirr + nloop) * N;
  gemm(CUBLAS_OP_N, N, nh, m, one, R.p, N, Q.p + size_t(m - nh) * m, m, zero, H, N);  // R Y
  for (int k = 0; k < nh; ++k) {
    const float sc = 1.f / std::sqrt(wh[size_t(m - nh + k)]);
    MTF_REQUIRE(cublasSscal(bh, N, &sc, H + size_t(k) * N, 1) == CUBLAS_STATUS_SUCCESS, MTF_ERR_CUDA,
                "cublasSscal failed");
  }
  MTF_CUDA(cudaStreamSynchronize(s));  // scratch is freed on return
}

// mesh-level eigenpairs of (D, G) for every block (once per mesh)
static void osrc_mesh_setup(mtf_mesh m, cudaStream_t s) {
  if (m->osrc_ready) return;
  const TriRule& rule = triangle_rule6();
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_os_s, rule.s, sizeof(rule.s), 0, cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_os_t, rule.t, sizeof(rule.t), 0, cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaMemcpyToSymbolAsync(c_os_w, rule.w, sizeof(rule.w), 0, cudaMemcpyHostToDevice, s));
  DevBuf<float> G;
  // padded offsets of the per-block W matrices
  m->osrc_off_h.assign(m->nd, 0);
  int64_t po = 0;
  for (int i = 0; i < m->nd; ++i) {
    m->osrc_off_h[i] = po;
    po += int64_t((m->blk[i].N + 3) & ~3) * m->blk[i].N;
  }
  m->d_osrc_off.upload(m->osrc_off_h, s);
  m->d_osrc_Vt.alloc(size_t(po));
  m->d_osrc_lam.alloc(size_t(m->n_rows));
  DevBuf<float> Dd;
  Dd.alloc(size_t(m->n_mat));
  G.alloc(size_t(m->n_mat));
  MTF_CUDA(cudaMemsetAsync(G.p, 0, size_t(m->n_mat) * sizeof(float), s));
  MTF_CUDA(cudaMemsetAsync(Dd.p, 0, size_t(m->n_mat) * sizeof(float), s));
  MTF_LAUNCH(KID_MISC, s, k_gram_divdiv<<<unsigned((m->n_bt + 127) / 128), 128, 0, s>>>(
      m->d_bt_v.p, m->d_bt_c.p, m->d_bt_area.p, m->d_bt_dof.p, m->d_bt_blk.p, m->d_blk_mat_off.p, m->d_blk_N.p,
      m->n_bt, G.p, Dd.p));
  SolverLease sl = solver_lease(s);  // held for the whole setup (osrc_harmonic takes the cuBLAS lock inside it)
  cusolverDnHandle_t h = sl.h;
  DevBuf<int> info;
  info.alloc(1);
  auto sygvd = [&](int N, float* A, float* B, float* W, const std::string& what) {
    int lwork = 0;
    MTF_REQUIRE(cusolverDnSsygvd_bufferSize(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                            N, A, N, B, N, W, &lwork) == CUSOLVER_STATUS_SUCCESS,
                MTF_ERR_CUDA, "cusolverDnSsygvd_bufferSize failed");
    DevBuf<float> work;
    work.alloc(size_t(std::max(lwork, 1)));
    MTF_REQUIRE(cusolverDnSsygvd(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, A, N, B,
                                 N, W, work.p, lwork, info.p) == CUSOLVER_STATUS_SUCCESS,
                MTF_ERR_CUDA, "cusolverDnSsygvd failed");
    int hinfo = 0;
    MTF_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    MTF_CUDA(cudaStreamSynchronize(s));
    MTF_REQUIRE(hinfo == 0, MTF_ERR_CUDA, "OSRC eigensolver failed for " + what + " (info " + std::to_string(hinfo) + ")");
  };
  // P1 Laplace-Beltrami pencils (S, M) per block
  DevBuf<float> S1, M1, mu, lam_tmp;
  S1.alloc(size_t(m->p1_nmat));
  M1.alloc(size_t(m->p1_nmat));
  mu.alloc(size_t(m->p1_nrow));
  lam_tmp.alloc(size_t(m->n_rows));
  MTF_CUDA(cudaMemsetAsync(S1.p, 0, S1.n * sizeof(float), s));
  MTF_CUDA(cudaMemsetAsync(M1.p, 0, M1.n * sizeof(float), s));
  MTF_LAUNCH(KID_MISC, s, k_p1_matrices<<<unsigned((m->n_bt + 127) / 128), 128, 0, s>>>(
      m->d_bt_v.p, m->d_bt_area.p, m->d_bt_lv.p, m->d_bt_blk.p, m->d_p1_off.p, m->d_p1_n.p, m->n_bt, S1.p, M1.p));
  DevBuf<float> Wtmp;
  for (int i = 0; i < m->nd; ++i) {
    const int N = m->blk[i].N, nv = m->p1_n[i];
    const int nirr = m->blk[i].T - 1, nloop = nv - 1;
    // a connected boundary of genus g: N = nirr + nloop + 2 g (Euler)
    const int nh = N - nirr - nloop;
    MTF_REQUIRE(nh >= 0 && nh % 2 == 0, MTF_ERR_MESH,
                "block-OSRC needs connected subdomain boundaries (Gamma_" + std::to_string(i) + ")");
    float* A = Dd.p + m->blk[i].mat_off;
    DevBuf<float> Gc;  // the mass matrix, kept for the harmonic fields
    if (nh > 0) {
      Gc.alloc(size_t(N) * N);
      MTF_CUDA(cudaMemcpyAsync(Gc.p, G.p + m->blk[i].mat_off, size_t(N) * N * sizeof(float),
                               cudaMemcpyDeviceToDevice, s));
    }
    sygvd(N, A, G.p + m->blk[i].mat_off, lam_tmp.p + m->blk[i].row_off, "the div-div pencil of block " + std::to_string(i));
    sygvd(nv, S1.p + m->p1_off_h[i], M1.p + m->p1_off_h[i], mu.p + m->p1_row_h[i],
          "the Laplace-Beltrami pencil of block " + std::to_string(i));
    // W = [irrotational eigenvectors, loop modes] -> Wtmp, then back into Vt
    Wtmp.alloc(size_t(N) * N);
    MTF_LAUNCH(KID_MISC, s, k_build_w<<<unsigned((int64_t(N) * N + 255) / 256), 256, 0, s>>>(
        A, lam_tmp.p + m->blk[i].row_off, S1.p + m->p1_off_h[i], mu.p + m->p1_row_h[i],
        m->d_edge_lohi.p + 2 * m->blk[i].row_off, m->d_edge_len.p + m->blk[i].row_off, N, nirr, nv, Wtmp.p,
        m->d_osrc_lam.p + m->blk[i].row_off));
    if (nh > 0) osrc_harmonic(N, nirr, nloop, nh, A, Gc.p, Wtmp.p, h, s);
    // padded row-major W^T (rows = modes), ld = N rounded up to 4: the
    // column-major W (rows = RWG dofs) with leading dimension ld
    const int ld = (N + 3) & ~3;
    MTF_LAUNCH(KID_MISC, s, k_pad_copy<<<unsigned((int64_t(N) * ld + 255) / 256), 256, 0, s>>>(
        Wtmp.p, N, ld, m->d_osrc_Vt.p + m->osrc_off_h[i]));
    MTF_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> nirr_h(m->nd);
  for (int i = 0; i < m->nd; ++i) nirr_h[i] = m->blk[i].T - 1;
  m->d_osrc_nirr.upload(nirr_h, s);
  // areas of Gamma_i for the damping parameter
  m->osrc_area.assign(m->nd, 0.0);
  for (int64_t q = 0; q < m->n_bt; ++q) m->osrc_area[m->bt_blk[q]] += m->bt_area[q];
  MTF_CUDA(cudaStreamSynchronize(s));
  m->osrc_ready = true;
}

// stream units of T~ (entry type 1: FP32, 3: FP16), built once per mesh
template <int ENT>
static const StreamUnits& ensure_os_units(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  StreamUnits& su = ENT == 3 ? m->os16_units : m->os_units;
  if (!su.ready) {
    std::vector<int64_t> ld(m->nd);
    for (int i = 0; i < m->nd; ++i) ld[i] = st_row_stride<ENT>(m->blk[i].N);
    build_stream_units(m, st_unit_rows<ENT>(), st_piece_len<ENT>(), st_eb<ENT>(),
                       ENT == 3 ? m->os16_off_h : m->os_T_off_h, ld, su, s);
  }
  return su;
}

// FP16 copy of T~ for the FP32 applies: block i is stored as T~_i / s_i
// (s_i = largest |re| or |im| of its entries, so every entry lies in
// [-1, 1] where FP16 keeps 11 significant bits), rows padded to a multiple
// of 4 entries; the combine's coefficients (rho, 1/rho) carry s_i.
static void osrc_half_copy(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  m->os16_off_h.assign(m->nd, 0);
  int64_t off = 0;
  for (int i = 0; i < m->nd; ++i) {
    m->os16_off_h[i] = off;
    off += int64_t(m->blk[i].N) * st_row_stride<3>(m->blk[i].N);
  }
  sys->d_osrc_T16.alloc(size_t(off));
  DevBuf<unsigned> mx;
  mx.alloc(size_t(m->nd));
  MTF_CUDA(cudaMemsetAsync(mx.p, 0, size_t(m->nd) * sizeof(unsigned), s));
  for (int i = 0; i < m->nd; ++i) {
    const int N = m->blk[i].N;
    const int64_t nn = int64_t(N) * st_row_stride<1>(N);
    MTF_LAUNCH(KID_MISC, s, k_os_absmax<<<unsigned(std::min<int64_t>(1024, (nn + 255) / 256)), 256, 0, s>>>(
        reinterpret_cast<const float2*>(sys->d_osrc_T.p) + m->os_T_off_h[i], nn, i, mx.p));
  }
  std::vector<unsigned> mh(static_cast<size_t>(m->nd));
  MTF_CUDA(cudaMemcpyAsync(mh.data(), mx.p, mh.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  std::vector<float> cf(static_cast<size_t>(4 * m->nd));
  for (int i = 0; i < m->nd; ++i) {
    float sc;
    std::memcpy(&sc, &mh[size_t(i)], sizeof(float));
    MTF_REQUIRE(std::isfinite(sc), MTF_ERR_NAN, "non-finite block-OSRC entries");
    if (!(sc > 0.f)) sc = 1.f;
    const int N = m->blk[i].N;
    const int ld16 = int(st_row_stride<3>(N));
    const int64_t nn = int64_t(N) * ld16;
    MTF_LAUNCH(KID_MISC, s, k_os_to_half<<<unsigned((nn + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float2*>(sys->d_osrc_T.p) + m->os_T_off_h[i], N, int(st_row_stride<1>(N)), ld16,
        1.f / sc, reinterpret_cast<__half2*>(sys->d_osrc_T16.p) + m->os16_off_h[i]));
    const double rr = sys->rho_re[i], ri = sys->rho_im[i], rn = rr * rr + ri * ri;
    cf[size_t(4 * i)] = float(sc * rr);
    cf[size_t(4 * i + 1)] = float(sc * ri);
    cf[size_t(4 * i + 2)] = float(sc * rr / rn);
    cf[size_t(4 * i + 3)] = float(-sc * ri / rn);
  }
  sys->d_os_coef16.upload(cf, s);
  std::vector<int64_t> ld16(static_cast<size_t>(m->nd));
  for (int i = 0; i < m->nd; ++i) ld16[size_t(i)] = st_row_stride<3>(m->blk[i].N);
  tc_build_osrc(sys, ld16, s);
  if (MTF_OSRC_TC) {
    // the tensor-core stream reads one contiguous run per unit
    const StreamUnits& su = ensure_os_units<3>(sys, s);
    sys->d_osrc_T16t.alloc(size_t(su.tiled_bytes / 4));
    tile_stream_operator(su, sys->d_osrc_T16.p, 4, sys->d_osrc_T16t.p, s);
  }
  MTF_CUDA(cudaStreamSynchronize(s));  // mx and the host tables go out of scope
}

void osrc_setup(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  osrc_mesh_setup(m, s);
  const int np = std::max(1, sys->opt.osrc_np);
  const double th = sys->opt.osrc_theta;
  using cd = std::complex<double>;
  // rotated-branch-cut Pade coefficients
  std::vector<double> pd(2 + 4 * np);
  const cd e = std::exp(cd(0, -th));
  cd R = 1.0;
  std::vector<double> a(np), b(np);
  for (int j = 1; j <= np; ++j) {
    a[j - 1] = 2.0 / (2 * np + 1) * std::pow(std::sin(j * M_PI / (2 * np + 1)), 2);
    b[j - 1] = std::pow(std::cos(j * M_PI / (2 * np + 1)), 2);
    R += a[j - 1] * (e - 1.0) / (1.0 + b[j - 1] * (e - 1.0));
  }
  const cd C0 = std::exp(cd(0, th / 2)) * R;
  pd[0] = C0.real();
  pd[1] = C0.imag();
  for (int j = 0; j < np; ++j) {
    const cd den = 1.0 + b[j] * (e - 1.0);
    const cd A = std::exp(cd(0, -th / 2)) * a[j] / (den * den);
    const cd B = e * b[j] / den;
    pd[2 + 4 * j] = A.real();
    pd[3 + 4 * j] = A.imag();
    pd[4 + 4 * j] = B.real();
    pd[5 + 4 * j] = B.imag();
  }
  std::vector<double> keps(2 * m->nd);
  for (int i = 0; i < m->nd; ++i) {
    const double k = sys->k_re[i];
    const double R = std::sqrt(m->osrc_area[i] / (4 * M_PI));
    keps[2 * i] = k;
    keps[2 * i + 1] = sys->opt.osrc_eps_scale * std::cbrt(k) * std::pow(R, -2.0 / 3.0);
  }
  DevBuf<double> d_pd, d_keps;
  d_pd.upload(pd, s);
  d_keps.upload(keps, s);
  sys->d_osrc_f.alloc(size_t(m->n_rows) * 2);
  MTF_LAUNCH(KID_MISC, s, k_osrc_symbol<<<unsigned((m->n_rows + 127) / 128), 128, 0, s>>>(
      m->d_osrc_lam.p, m->d_row_blk.p, m->n_rows, m->d_blk_row_off.p, m->d_osrc_nirr.p, sys->d_k.p, d_keps.p,
      d_pd.p, np, sys->opt.osrc_type == 2 ? 1 : 0, reinterpret_cast<float2*>(sys->d_osrc_f.p)));
  // T~ rows padded to an even length (8-byte entries: 16-byte aligned rows)
  m->os_T_off_h.assign(m->nd, 0);
  int64_t toff = 0;
  for (int i = 0; i < m->nd; ++i) {
    m->os_T_off_h[i] = toff;
    toff += int64_t(m->blk[i].N) * (m->blk[i].N + (m->blk[i].N & 1));
  }
  sys->d_osrc_T.alloc(size_t(toff) * 2);
  // T~_i = W_i diag(f_i) W_i^T on the tensor cores
  osrc_form_tc(sys, s);
  if (sys->opt.osrc_half) osrc_half_copy(sys, s);
  osrc_prepare_fp64_apply(sys, s);
  MTF_CUDA(cudaStreamSynchronize(s));  // scratch and d_pd / d_keps are freed on return
}

template <int NC, class ZT, bool ADJ = false, int ENT = 1>
static void os_launch(mtf_system sys, const float* r32, int64_t ldr, ZT* z, int64_t ldz, int c0, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const StreamUnits& su = ENT == 3 ? m->os16_units : m->os_units;
  const void* ent = ENT == 3 ? static_cast<const void*>(sys->d_osrc_T16.p) : static_cast<const void*>(sys->d_osrc_T.p);
  const float* cf = ENT == 3 ? sys->d_os_coef16.p : sys->d_rho32.p;
  if (ENT == 3 && MTF_OSRC_TC)
    launch_stream_tc<NC>(sys, sys->d_osrc_T16t.p, su, r32, ldr, c0, sys->d_os_part.p, KID_OSRC, s);
  else
    launch_stream_tiles<NC, ENT>(sys, ent, su, r32, ldr, c0, sys->d_os_part.p, KID_OSRC, s);
  MTF_LAUNCH(KID_OSCOMBINE, s,
             launch_pdl(k_os_combine<NC, ZT, ADJ, ENT>, dim3(unsigned((m->n_rows * 32 + 255) / 256)), dim3(256), 0,
                        s, sys->d_os_part.p, su.pmax, m->d_row_blk.p, m->d_blk_N.p, m->d_blk_dof_off.p,
                        m->d_blk_row_off.p, sys->d_rho.p, cf, z, ldz, c0, m->n_rows));
}

template <class ZT, bool ADJ, int ENT>
static void osrc_stream_ent(mtf_system sys, const float* r32, int64_t ldr, ZT* z, int64_t ldz, int nrhs,
                            cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const StreamUnits& su = ensure_os_units<ENT>(sys, s);
  const size_t npart = size_t(m->n_rows) * su.pmax * 16;
  if (sys->d_os_part.n < npart) sys->d_os_part.alloc(npart);
  for (int c0 = 0; c0 < nrhs; c0 += 4) {
    const int nc = std::min(4, nrhs - c0);
    if (nc == 1) os_launch<1, ZT, ADJ, ENT>(sys, r32, ldr, z, ldz, c0, s);
    else if (nc == 2) os_launch<2, ZT, ADJ, ENT>(sys, r32, ldr, z, ldz, c0, s);
    else if (nc == 3) os_launch<3, ZT, ADJ, ENT>(sys, r32, ldr, z, ldz, c0, s);
    else os_launch<4, ZT, ADJ, ENT>(sys, r32, ldr, z, ldz, c0, s);
  }
}

// FP32 output follows the system's osrc_half option (FP16 copy of T~);
// FP64 output always streams the FP32 T~
template <class ZT, bool ADJ = false>
static void osrc_stream(mtf_system sys, const float* r32, int64_t ldr, ZT* z, int64_t ldz, int nrhs, cudaStream_t s) {
  stream_prepare(sys, s);
  if constexpr (sizeof(ZT) == 4) {
    if (!ADJ && tc_wide_apply(sys, nrhs) && tc_osrc_enabled(sys)) {
      launch_osrc_apply_tc(sys, r32, ldr, z, ldz, nrhs, s);
      return;
    }
    if (sys->opt.osrc_half) {
      osrc_stream_ent<ZT, ADJ, 3>(sys, r32, ldr, z, ldz, nrhs, s);
      return;
    }
  }
  osrc_stream_ent<ZT, ADJ, 1>(sys, r32, ldr, z, ldz, nrhs, s);
}

void launch_osrc_apply(mtf_system sys, const double* r, int64_t ldr, double* z, int64_t ldz, int nrhs,
                       cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  const int64_t n2 = 2 * m->n_total;
  if (sys->d_osrc_r32.n < size_t(n2) * nrhs) sys->d_osrc_r32.alloc(size_t(n2) * nrhs);
  MTF_LAUNCH(KID_OSRC, s, k_to_f32_cols<<<unsigned((n2 * nrhs + 255) / 256), 256, 0, s>>>(r, ldr, n2, nrhs, sys->d_osrc_r32.p));
  osrc_stream<double>(sys, sys->d_osrc_r32.p, m->n_total, z, ldz, nrhs, s);
}

// Everything the FP64-output apply keeps per system or mesh (the error word
// and grid size of the streaming kernels, the FP32 T~ stream units, the
// per-row piece sums), set up at assembly so that
// launch_osrc_apply_prepared allocates nothing.
void osrc_prepare_fp64_apply(mtf_system sys, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  stream_prepare(sys, s);
  const StreamUnits& su = ensure_os_units<1>(sys, s);
  const size_t npart = size_t(m->n_rows) * su.pmax * 16;
  if (sys->d_os_part.n < npart) sys->d_os_part.alloc(npart);
}

// launch_osrc_apply with the FP32 copy of r written to the caller's r32
// (2 n_total nrhs floats); needs osrc_prepare_fp64_apply (done by every
// block-OSRC assembly) and allocates nothing.
void launch_osrc_apply_prepared(mtf_system sys, const double* r, int64_t ldr, double* z, int64_t ldz, int nrhs,
                                float* r32, cudaStream_t s) {
  mtf_mesh m = sys->mesh;
  MTF_REQUIRE(m->os_units.ready && sys->d_mv_ctl.p && sys->mv_grid > 0 &&
                  sys->d_os_part.n >= size_t(m->n_rows) * m->os_units.pmax * 16,
              MTF_ERR_ARG, "block-OSRC apply tables are not prepared (system not assembled with block-OSRC)");
  const int64_t n2 = 2 * m->n_total;
  MTF_LAUNCH(KID_OSRC, s, k_to_f32_cols<<<unsigned((n2 * nrhs + 255) / 256), 256, 0, s>>>(r, ldr, n2, nrhs, r32));
  osrc_stream<double>(sys, r32, m->n_total, z, ldz, nrhs, s);
}

// FP32 in, FP32 out (the FP32-basis inner solver)
void launch_osrc_apply_f32(mtf_system sys, const float* r, int64_t ldr, float* z, int64_t ldz, int nrhs,
                           cudaStream_t s) {
  osrc_stream<float>(sys, r, ldr, z, ldz, nrhs, s);
}

// w -> P^H w (FP32): the adjoint of the block-OSRC operator, used to
// back-propagate through preconditioned products
void launch_osrc_apply_adj_f32(mtf_system sys, const float* w, int64_t ldw, float* z, int64_t ldz, int nrhs,
                               cudaStream_t s) {
  const int64_t n = sys->mesh->n_total;
  if (sys->d_os_adj32.n < size_t(2 * n) * nrhs) sys->d_os_adj32.alloc(size_t(2 * n) * nrhs);
  launch_conj32(w, ldw, n, nrhs, sys->d_os_adj32.p, n, s);
  osrc_stream<float, true>(sys, sys->d_os_adj32.p, n, z, ldz, nrhs, s);
}

}  // namespace mtf
