// Internal declarations of libmtf (not part of the public C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mtf.h"
#include "stream_plan.h"

namespace mtf {

// ---------------------------------------------------------------------------
// errors: thrown inside the library, turned into mtf_status at the C-ABI
// ---------------------------------------------------------------------------
struct Error {
  mtf_status status;
  std::string msg;
};

void set_last_error(const std::string& msg);

#define MTF_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::mtf::Error{e_ == cudaErrorMemoryAllocation ? MTF_ERR_OOM : MTF_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_)};      \
  } while (0)

#define MTF_REQUIRE(cond, st, msg)                      \
  do {                                                  \
    if (!(cond)) throw ::mtf::Error{(st), (msg)};       \
  } while (0)

// Owning device buffer.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count == n && p) return;
    release();
    if (count == 0) return;
    MTF_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void upload(const std::vector<T>& h, cudaStream_t s) {
    alloc(h.size());
    if (!h.empty()) MTF_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
};

// ---------------------------------------------------------------------------
// quadrature tables (generated on the host from their defining equations)
// ---------------------------------------------------------------------------
struct TriRule {
  double s[6], t[6], w[6];  // reference triangle {s,t>=0, s+t<=1}, sum w = 1/2
};
const TriRule& triangle_rule6();
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
// Sauter-Schwab rule: (x1, x2, y1, y2, w) per point, kinds 0 coincident,
// 1 common edge, 2 common vertex.
void sauter_schwab_rule(int kind, int n, std::vector<double>& pts);

// ---------------------------------------------------------------------------
// mesh (Algorithm 1 and RWG tables)
// ---------------------------------------------------------------------------
struct BlockInfo {
  int32_t T = 0;          // triangles of Gamma_i
  int32_t N = 0;          // RWG dofs of Gamma_i
  int64_t bt_off = 0;     // first block-triangle index
  int64_t dof_off = 0;    // unknown offset 2 sum_{j<i} N_j
  int64_t mat_off = 0;    // first dense entry of the block's matrices
  int64_t row_off = 0;    // first exchange row (sum_{j<i} N_j)
};

// Singular pair record (device): block-triangle ids and the Sauter-Schwab
// vertex orders (local vertex indices 0..2 packed in 2 bits each).
struct SingPair {
  int32_t tau;   // block-triangle index of the test triangle
  int32_t sig;   // block-triangle index of the trial triangle
  int32_t block;
  int32_t code;  // kind (bits 0-1) | perm_tau (bits 2-7) | perm_sig (bits 8-13)
};

// Exchange (transmission Gram) entry: row = (block i, dof m); 6 entries per
// row, one per (triangle of Gamma_i containing edge m, local edge b of the
// neighbour's RWG function on that triangle).
struct XEntry {
  int32_t bt_i;   // block-triangle of the row's triangle in block i
  int32_t bt_j;   // the same skeleton triangle seen from block j
  int32_t col;    // global unknown index of the D slot of dof_j(t, b)
  int32_t ab;     // a | (b << 2) | (nj << 4): local edges and N_j for the N slot offset
};

// Work units of a bulk-copy tiled streaming operator apply (stream.cuh):
// groups of consecutive rows of a block x one column piece, piece-major
// within a block.  units: {N_i, global row of the first row, first input
// column, len | piece << 12 | rows << 24 (rows <= 31)}; src: first entry of
// the first row's piece in the stored operator.
struct StreamUnits {
  bool ready = false;
  int64_t n_units = 0;
  int32_t pmax = 1;
  DevBuf<int4> d_units;
  DevBuf<int64_t> d_src;
  // tiled copy of the operator (one contiguous run per unit): byte offset of
  // every unit and the total size
  DevBuf<int64_t> d_toff;
  int64_t tiled_bytes = 0;
};



}  // namespace mtf

struct mtf_mesh_s {
  int32_t nv = 0, nt = 0, nd = 0;
  bool uploaded = false;                     // device copies made at the first mtf_assemble
  std::vector<double> V;
  std::vector<int32_t> F, L;                 // canonical: normal from min to max label
  std::vector<mtf::BlockInfo> blk;
  int64_t n_total = 0, n_rows = 0, n_bt = 0, n_mat = 0;
  int64_t pair_counts[4] = {0, 0, 0, 0};    // coincident, edge, vertex, regular
  // host copies of the per-block-triangle tables
  std::vector<int32_t> bt_tri, bt_dof, bt_vid, bt_blk;
  std::vector<int8_t> bt_swap;
  std::vector<double> bt_v, bt_c, bt_area;
  std::vector<mtf::SingPair> sing;
  std::vector<mtf::XEntry> xent;
  std::vector<int32_t> dof_bt;               // per exchange row: 2 x (bt*3 + a)
  // device copies
  mtf::DevBuf<double> d_bt_v, d_bt_c, d_bt_area;
  mtf::DevBuf<int32_t> d_bt_dof, d_bt_vid, d_bt_blk, d_dof_bt;
  mtf::DevBuf<int8_t> d_bt_swap;
  mtf::DevBuf<mtf::SingPair> d_sing;
  mtf::DevBuf<mtf::XEntry> d_xent;
  mtf::DevBuf<int64_t> d_blk_mat_off;        // per block
  mtf::DevBuf<int32_t> d_blk_N, d_blk_T;
  mtf::DevBuf<int64_t> d_blk_bt_off, d_blk_dof_off, d_blk_row_off;
  std::vector<int64_t> reg_cta_prefix;       // regular-pair CTA prefix over blocks
  mtf::DevBuf<int64_t> d_reg_cta_prefix;
  mtf::DevBuf<int32_t> d_row_blk;            // exchange row -> block
  // streaming work units of the FP32 matvec ({T, K} entries) and of the
  // OSRC apply (T~ entries)
  mtf::StreamUnits mv_units, os_units;
  std::vector<int64_t> os_T_off_h;           // first entry of each block's T~ (rows of even stride)
  std::vector<int64_t> os16_off_h;           // first entry of each block's FP16 T~ (rows padded to 4 entries)
  mtf::StreamUnits os16_units;               // stream units of the FP16 T~
  // block-OSRC: eigenpairs of (div-div, mass) per block, computed once
  bool osrc_ready = false;
  mtf::DevBuf<float> d_osrc_Vt, d_osrc_lam;              // W^T (per block, padded rows), |xi|^2 per mode
  mtf::DevBuf<int32_t> d_osrc_nirr;                      // irrotational modes per block
  std::vector<int64_t> osrc_off_h;                       // padded W offsets per block
  mtf::DevBuf<int64_t> d_osrc_off;
  std::vector<double> osrc_area;
  // P1 (vertex) tables of every Gamma_i for the loop modes
  std::vector<int32_t> p1_n;                             // vertices of Gamma_i
  std::vector<int64_t> p1_off_h, p1_row_h;               // dense (V_i^2) and row offsets
  int64_t p1_nmat = 0, p1_nrow = 0;
  std::vector<int32_t> bt_lv;                            // local vertex index per triangle corner
  std::vector<int32_t> edge_lohi;                        // per exchange row: local (lo, hi) vertex
  std::vector<double> edge_len;                          // per exchange row: edge length
  mtf::DevBuf<int32_t> d_bt_lv, d_p1_n, d_edge_lohi;
  mtf::DevBuf<int64_t> d_p1_off;
  mtf::DevBuf<double> d_edge_len;
};

namespace mtf {
struct GmresWork;
struct Gmres32Work;
struct BlockWork;
struct TcMatvec;
struct TtForm;
struct LearnedState;
}

struct mtf_system_s {
  mtf_mesh mesh = nullptr;
  mtf_options opt{};
  // host time of the inner block FGMRES steps of the current solve (s)
  double t_launch = 0, t_lsq = 0, t_wait = 0;
  double k0 = 0;
  std::vector<double> k_re, k_im, rho_re, rho_im;
  mtf::DevBuf<double> d_k, d_rho;            // (re, im) per block
  mtf::DevBuf<double> d_wdir, d_wpol, d_brhs;  // mtf_solve: wave parameters and right-hand sides (kept)
  mtf::DevBuf<double> d_TK64;                // FP64: 4 doubles per dense entry
  mtf::DevBuf<float> d_TK64hl;               // residual_fp64: the FP64 entries as FP32 pairs (all hi, then all lo)
  mtf::DevBuf<float> d_TK32;                 // mixed: 4 floats per dense entry
  mtf::DevBuf<float> d_TK32t;                // the same, tiled per stream unit (streaming matvec)
  mtf::DevBuf<double> d_xval;                // exchange values (6 per row)
  mtf::DevBuf<float> d_xval32;               // FP32 copy of the exchange values
  mtf::DevBuf<float> d_rho32;                // per block: rho (re, im), 1 / rho (re, im)
  mtf::DevBuf<double> d_ss_pts[3];           // Sauter-Schwab tables
  // FP32 geometry of the mixed regular-pair kernel (per block-triangle)
  mtf::DevBuf<float> d_x32;                  // FP32 copy of the matvec input (mixed path)
  mtf::DevBuf<float> d_adj32;                // conjugated input of the adjoint matvec
  mtf::DevBuf<float> d_os_adj32;             // conjugated input of the adjoint block-OSRC apply
  mtf::DevBuf<float> d_osrc_f, d_osrc_r32;   // OSRC symbol (complex) and apply scratch
  mtf::DevBuf<float> d_osrc_T;               // complex T~ of every block (rows of N_i, at the blocks' mat_off)
  mtf::DevBuf<uint32_t> d_osrc_T16;          // FP16 (__half2) copy of T~, scaled per block (osrc_half)
  mtf::DevBuf<uint32_t> d_osrc_T16t;         // the same, tiled per stream unit (tensor-core stream)
  mtf::DevBuf<float> d_os_coef16;            // per block: s_i (rho, 1/rho) for the FP16 copy
  mtf::DevBuf<float> d_os_part;              // per-row piece sums of the OSRC apply
  mtf::DevBuf<double> d_cen;
  mtf::DevBuf<float> d_qx, d_qw, d_pv, d_cc;
  int32_t ss_npts[3] = {0, 0, 0};
  // streaming matvec: per-row piece sums and the error word (d_mv_ctl[2])
  mtf::DevBuf<float> d_mv_part;
  mtf::DevBuf<unsigned> d_mv_ctl;
  int32_t mv_grid = 0;
  mtf::GmresWork* gw = nullptr;
  mtf::Gmres32Work* gw32 = nullptr;
  mtf::BlockWork* bw = nullptr;          // block FGMRES workspace (block32.cu)
  mtf::TcMatvec* tc = nullptr;           // tensor-core matvec tables and operator copy (mv_tc.cu)
  mtf::TtForm* tt = nullptr;             // tensor-core block-OSRC formation (osrc_form_tc.cu)
  mtf::LearnedState* learned = nullptr;  // learned OSRC correction (learned.cu)
  bool learned_active = false;           // used by the current solve (cleared by its fallback)
};

namespace mtf {
// kernel ids of the per-kernel accounting (profile.cpp)
enum KernelId {
  KID_REGULAR64 = 0, KID_SINGULAR64, KID_XVALUES, KID_RHS, KID_MATVEC64, KID_DOTS, KID_AXPY,
  KID_NORM, KID_SUB, KID_FARFIELD, KID_SPLIT, KID_REGULAR32, KID_MATVEC32, KID_OSRC, KID_MLP,
  KID_MISC, KID_MVCOMBINE, KID_OSCOMBINE, KID_MVTC, KID_MVTC_PREP, KID_MVTC_COMBINE, KID_TC_TILE,
  KID_BCHOL, KID_BXFORM, KID_BSTORE, KID_TT, KID_TT_MMA, KID_TCA_PREP, KID_BGRAM, KID_COUNT
};
void prof_begin(int kid, cudaStream_t s);
void prof_end(int kid, cudaStream_t s);
void prof_enable(bool on);
void prof_read(int n, int64_t* launches, double* ms, double* bytes = nullptr);
// algorithmic bytes of a launch (each stored operator entry, input and
// output value counted once), summed per kernel id for the roofline
void prof_bytes(int kid, double b);
const char* kernel_name(int kid);
// launch a kernel with accounting: LAUNCH(kid, stream, kernel<<<...>>>(args))
#define MTF_LAUNCH(kid, stream, ...)          \
  do {                                        \
    ::mtf::prof_begin((kid), (stream));       \
    __VA_ARGS__;                              \
    MTF_CUDA(cudaGetLastError());             \
    ::mtf::prof_end((kid), (stream));         \
  } while (0)

// Programmatic dependent launch for the chains of short kernels of the
// inner solver: a kernel launched by launch_pdl may be scheduled before its
// predecessor on the stream has finished; its first statements must be
// MTF_PDL_WAIT() (returns once the predecessor grid has completed and its
// memory is visible, so stream order holds for every access) and
// MTF_PDL_TRIGGER() (lets the next such kernel be scheduled once all CTAs of
// this one have started).  Both are no-ops for ordinary launches.
#define MTF_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
#define MTF_PDL_TRIGGER() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  MTF_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

void assemble_into(mtf_system sys, double k0, const double* eps_r, const double* mu_r, cudaStream_t s);
// kernels launched from the host side (implemented in the .cu files)
void launch_assemble(mtf_system sys, cudaStream_t s);
void launch_assemble_regular32(mtf_system sys, cudaStream_t s);
void osrc_setup(mtf_system sys, cudaStream_t s);
// z = A~ r (block-OSRC, Eq. 19); column c of r (z) at r + 2 c ldr (z + 2 c ldz)
void launch_osrc_apply(mtf_system sys, const double* r, int64_t ldr, double* z, int64_t ldz, int nrhs,
                       cudaStream_t s);
void launch_osrc_apply_f32(mtf_system sys, const float* r, int64_t ldr, float* z, int64_t ldz, int nrhs,
                           cudaStream_t s);
// set-up of the FP64-output apply done at every block-OSRC assembly, and the
// apply itself with the FP32 copy of r in the caller's r32 (2 n_total nrhs
// floats): allocates nothing
void osrc_prepare_fp64_apply(mtf_system sys, cudaStream_t s);
void launch_osrc_apply_prepared(mtf_system sys, const double* r, int64_t ldr, double* z, int64_t ldz, int nrhs,
                                float* r32, cudaStream_t s);
// Streaming matvec of the FP32-stored operator (matvec32.cu).  The dense
// part reads the FP32 vector x32 (column stride ld32, complex units); the
// exchange rows read x.  f32: FP32 in and out.
void launch_matvec_f32(mtf_system sys, const float* x, int64_t ldx, float* y, int64_t ldy, int nrhs,
                       cudaStream_t s);
void launch_matvec_stream64(mtf_system sys, const double* x, int64_t ldx, const float* x32, int64_t ld32, double* y,
                            int64_t ldy, int nrhs, cudaStream_t s);
// y = M^H v (FP32), with T and K taken as complex symmetric (their Galerkin
// forms are, and the assembly keeps them so to rounding)
void launch_matvec_adj_f32(mtf_system sys, const float* v, int64_t ldv, float* y, int64_t ldy, int nrhs,
                           cudaStream_t s);
// z = P^H w (FP32), the adjoint of the block-OSRC operator
void launch_osrc_apply_adj_f32(mtf_system sys, const float* w, int64_t ldw, float* z, int64_t ldz, int nrhs,
                               cudaStream_t s);
// out^c = conj(v^c) over n complex entries
void launch_conj32(const float* v, int64_t ldv, int64_t n, int ncols, float* out, int64_t ldo, cudaStream_t s);
void check_matvec_stream(mtf_system sys, cudaStream_t s);
// grid size and error word shared by the streaming kernels
void stream_prepare(mtf_system sys, cudaStream_t s);
// fill u with the units of the tiled streaming kernel: every block's rows in
// groups of `rows`, cut into pieces of at most piece_len entries (lengths and
// starts multiples of 16 / entry_bytes); blk_entry_off[i] = first entry of
// block i, row_stride[i] = entries between its rows.  Checks that every bulk
// copy of the units is 16-byte aligned.
void build_stream_units(mtf_mesh m, int rows, int piece_len, int entry_bytes, const std::vector<int64_t>& blk_entry_off,
                        const std::vector<int64_t>& row_stride, StreamUnits& u, cudaStream_t s);
// tiled copy (su.tiled_bytes) of a streamed operator with eb-byte entries
void tile_stream_operator(const StreamUnits& su, const void* dense, int eb, void* tiled, cudaStream_t s);
void tile_matvec_operator(mtf_system sys, cudaStream_t s);
// One FGMRES cycle of the mixed path on M d = r from d = 0 (FP32 Krylov
// basis, FP64 reductions), then x += d.  Stops when every right-hand side's
// estimate reaches tol relative to ||r|| (reached = true), after the restart
// length or after max_iter iterations; iters[c] += iterations of rhs c.
// cycle: index of the cycle within the solve.  With opt.recycle, cycle 0
// keeps its Krylov space (C = M U) and cycle 1 starts from it (GCRO): the
// residual is projected out of C and the new basis is orthogonalised
// against C, so the second cycle does not repeat the first one's slow
// start.
mtf_status fgmres_cycle32(mtf_system sys, int nrhs, const double* r_dev, double* x_dev, double tol, int max_iter,
                          std::vector<int>& iters, bool& reached, cudaStream_t s, int cycle);
// matvec flavours: storage / accumulation precision
enum MatvecKind { MV_AUTO = 0, MV_FP64 = 1, MV_FP32 = 2, MV_FP32_ACC64 = 3 };
void launch_matvec_kind(mtf_system sys, int kind, const double* x, int64_t ldx, double* y, int64_t ldy,
                        int nrhs, cudaStream_t s);
void launch_exchange_values(mtf_system sys, cudaStream_t s);
// y = M x; column c of x (y) starts at x + 2 c ldx (y + 2 c ldy) doubles.
void launch_matvec(mtf_system sys, const double* x, int64_t ldx, double* y, int64_t ldy, int nrhs,
                   cudaStream_t s);
void launch_rhs(mtf_system sys, int nrhs, const double* d_dirs, const double* d_pols, double* b,
                cudaStream_t s);
void launch_farfield(mtf_system sys, const double* x, int nrhs, const double* d_obs, int nobs,
                     double* f, cudaStream_t s);
// U(x) by the representation formula (Eq. 8) at npts points (device, 3 each)
// in the subdomains d_dom (device), from the solutions x; f: device complex128
// (nrhs x npts x 3)
void launch_nearfield(mtf_system sys, const double* x, int nrhs, const double* d_pts, const int32_t* d_dom,
                      int npts, double* f, cudaStream_t s);
void launch_get_block(mtf_system sys, int i, double* t_out, double* k_out, cudaStream_t s);
mtf_status solve(mtf_system sys, int nrhs, const double* b_dev, double* x_dev, mtf_solve_stats* st,
                 cudaStream_t s);
void destroy_gmres(GmresWork* w);
void destroy_gmres32(Gmres32Work* w);
void destroy_block32(BlockWork* w);
void destroy_tc(TcMatvec* t);
void destroy_tt(TtForm* t);

// right-hand sides of one pass of the FMA streaming applies; wider applies
// go to the tensor cores (mv_tensor)
constexpr int kFmaPassRhs = 4;
// whether an apply to nrhs right-hand sides runs on the tensor cores (more
// than one FMA pass, tensor-core tables built, not overridden by the
// autotuner), and the autotuner's plan setter (mv_tc.cu)
bool tc_wide_apply(mtf_system sys, int nrhs);
void tc_set_plan(mtf_system sys, int waves, int min_len, int grid, bool prefer_fma, cudaStream_t s);
// FP32, FP64 FLOP/s and SFU results per second of the device (probe.cu)
void probe_peaks(double* rates, cudaStream_t s);
// T~_i = W_i diag(f_i) W_i^T of every block into sys->d_osrc_T on the tensor
// cores (osrc_form_tc.cu)
void osrc_form_tc(mtf_system sys, cudaStream_t s);
// tensor-core matvec (mv_tc.cu): the FP16 hi / lo tiled operator copy built
// after every mixed assembly (opt.mv_tensor), and y = M x from it
void tc_build_operator(mtf_system sys, cudaStream_t s);
bool tc_matvec_enabled(mtf_system sys);
void launch_matvec_tc(mtf_system sys, const float* x, int64_t ldx, float* y, int64_t ldy, int nrhs, cudaStream_t s);
// block-OSRC on the tensor cores from the FP16 T~ (mv_tc.cu)
// (ld16: per block, the row stride of the FP16 T~ copy in entries)
void tc_build_osrc(mtf_system sys, const std::vector<int64_t>& ld16, cudaStream_t s);
bool tc_osrc_enabled(mtf_system sys);
void launch_osrc_apply_tc(mtf_system sys, const float* r, int64_t ldr, float* z, int64_t ldz, int nrhs,
                          cudaStream_t s);
// One block flexible GMRES cycle of the mixed path on M D = R from D = 0 for
// the s right-hand sides together (block32.cu): one Krylov space of blocks of
// s vectors, FP32 basis, FP64 Hessenberg sums; x += D.  Stops when every
// right-hand side's estimate reaches tol relative to its ||r|| (reached =
// true), after opt.restart block steps, after max_iter block steps or when
// every direction is deflated; iters[c] += block steps.
mtf_status fgmres_block32(mtf_system sys, int s, const double* r_dev, double* x_dev, double tol, int max_iter,
                          std::vector<int>& iters, bool& reached, cudaStream_t st);
void destroy_learned(LearnedState* l);
// learned OSRC correction (learned.cu)
int64_t learned_param_count(mtf_system sys);
void learned_init(mtf_system sys, int kind, uint64_t seed, cudaStream_t s);
int learned_kind(mtf_system sys);
void learned_set_params(mtf_system sys, const float* host, cudaStream_t s);
void learned_get_params(mtf_system sys, float* host, cudaStream_t s);
void learned_features(mtf_system sys, float* X, cudaStream_t s);
void learned_loss_grad(mtf_system sys, const float* X, const float* T, const float* w, int64_t rows, float* grad_out,
                       double* loss_host, cudaStream_t s);
void learned_apply_inplace(mtf_system sys, const float* r, int64_t ldr, float* z, int64_t ldz, int nrhs,
                           cudaStream_t s);
void learned_stencil_adjoint(mtf_system sys, const float* w, float* out_r, float* out_p, int nrhs, cudaStream_t s);
void learned_power_grad(mtf_system sys, const float* Z, int pb, double c0r, double c0i, int K, float* grad_out,
                        double* loss_host, cudaStream_t s);
double learned_centre(mtf_system sys, double* im, cudaStream_t s);
void learned_train(mtf_system sys, int steps, double lr, int batch, int K, uint64_t seed, double* loss_first,
                   double* loss_last, cudaStream_t s);
}  // namespace mtf
