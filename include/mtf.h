/*
 * libmtf -- local multiple traces formulation (MTF) for time-harmonic
 * Maxwell transmission problems through heterogeneous scatterers, on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2502.10907 ("Local Multiple Traces Formulation for
 * Heterogeneous Electromagnetic Scattering: Implementation and
 * Preconditioning").  Each entry point cites the passage that defines what it
 * computes.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Complex numbers are interleaved (re, im) pairs.  "complex128" = two
 *   doubles, "complex64" = two floats.
 * - Unknown vector layout (Sec. 3.2, Eq. 16): blocks i = 0..M in order; block
 *   i holds [D coefficients (N_i), N coefficients (N_i)] of
 *   u_i = (gamma_D E, rho_i gamma_N E) in the RWG basis of Gamma_i; block
 *   offsets are 2 * sum_{j<i} N_j.  Multi-vector arguments are column-major
 *   n_total x nrhs (column c starts at c * n_total).
 * - RWG dofs of Gamma_i are the edges of Gamma_i ordered by increasing
 *   (lower vertex id, higher vertex id); the RWG function of edge e on
 *   triangle t of Gamma_i is s * l / (2 A) (x - v) with v the vertex opposite
 *   e, l = |e|, A = area(t), s = dir(e, t) * swap_i(t), dir = +1 iff t's
 *   vertex order runs along e from the lower to the higher vertex id.
 * - Ownership: the caller owns every pointer it passes; host inputs are
 *   copied before the call returns.  Handles own their device memory.
 * - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *   default stream).  Device work is enqueued on it; calls that return
 *   host-side results (stats, info) synchronise it.
 * - Errors: every call returns an mtf_status and never throws.  On error the
 *   output buffers are unspecified and handles remain valid; mtf_last_error()
 *   describes the last failure of the calling thread.
 * - Device pointers must be 16-byte aligned.
 */
#ifndef MTF_H_
#define MTF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mtf_mesh_s* mtf_mesh;
typedef struct mtf_system_s* mtf_system;

typedef enum {
  MTF_OK = 0,
  MTF_ERR_ARG = 1,      /* invalid argument (null pointer, size, range)      */
  MTF_ERR_MESH = 2,     /* skeleton mesh violates the admissibility rules    */
  MTF_ERR_CUDA = 3,     /* a CUDA runtime call failed                        */
  MTF_ERR_OOM = 4,      /* device allocation failed                          */
  MTF_ERR_NOCONV = 5,   /* solver reached max_iter above the tolerance       */
  MTF_ERR_NAN = 6,      /* non-finite value met in the solver                */
  MTF_ERR_TIMEOUT = 7   /* a bounded device wait ran out                     */
} mtf_status;

typedef enum {
  MTF_PREC_FP64 = 0,    /* FP64 assembly, storage, matvec and solver         */
  MTF_PREC_MIXED = 1    /* FP32 regular pairs + FP32 storage / matvec, FP64
                           singular pairs, FP64 Hessenberg sums, FP64
                           iterate with double-float (or, with
                           residual_df = 0, FP64) refinement residuals       */
} mtf_precision;

typedef enum {
  MTF_PRECOND_NONE = 0,
  MTF_PRECOND_OSRC = 1  /* block-OSRC of Sec. 4.4 (Eq. 19)                   */
} mtf_precond;

typedef struct {
  int32_t precision;    /* mtf_precision, default MTF_PREC_FP64              */
  int32_t n_ss;         /* Gauss points per coordinate of the Sauter-Schwab
                           rules (default 4, range 1..12)                     */
  int32_t restart;      /* GMRES restart length m (default 100)              */
  int32_t max_iter;     /* total GMRES iterations per solve (default 2000)   */
  double tol;           /* relative residual ||b - M x|| / ||b|| target
                           (default 1e-5, Sec. 5.3)                           */
  int32_t precond;      /* mtf_precond, default MTF_PRECOND_NONE             */
  int32_t osrc_np;      /* Pade order N_p of the OSRC square root (default 4)*/
  double osrc_theta;    /* branch-cut rotation angle (default pi/2)          */
  double osrc_eps_scale;/* damping eps = osrc_eps_scale k^(1/3) R^(-2/3)
                           with R the block's radius (default 0.39)          */
  int32_t max_refine;   /* mixed mode: outer FP64 refinement steps whose
                           FP32 inner solve reached its tolerance (default 4);
                           inner cycles that end on the restart length are
                           restarts and count against max_iter only          */
  int32_t learned;      /* 1: mtf_solve adds the trained learned correction
                           to block-OSRC (mixed precision with
                           MTF_PRECOND_OSRC only; see mtf_learned_init);
                           default 0                                         */
  int32_t osrc_half;    /* 1: the FP32 block-OSRC applies (the mixed inner
                           solver, mtf_precond_apply_f32) stream an FP16 copy
                           of T~ scaled per block (relative entry error
                           <= 2^-11 of the block's largest entry; the solution
                           is unaffected, FGMRES uses the vectors applied);
                           0: FP32 T~.  Default 1                            */
  int32_t recycle;      /* 1: in the mixed path the second inner FGMRES cycle
                           of a per-rhs solve reuses the first cycle's Krylov
                           space (GCRO-style: the new residual is projected
                           out of it and new basis vectors are orthogonalised
                           against it) instead of restarting from scratch;
                           0: plain restart.  The block solver
                           (block_krylov) always starts a cycle afresh.
                           Default 1                                         */
  int32_t residual_df;  /* mixed mode: 1: the outer refinement residuals
                           b - M x apply the FP32-stored operator to the FP64
                           iterate in double-float arithmetic (iterate split
                           into FP32 pairs, error-free products and sums;
                           about 2^-46 relative, on the FP32 pipes);
                           0: FP64 products and sums.  Default 1             */
  int32_t block_krylov; /* mixed mode with nrhs >= 4: 1: the inner FGMRES
                           cycles build one block Krylov space shared by all
                           right-hand sides (block flexible GMRES, block
                           classical Gram-Schmidt twice with the second pass
                           lagged one step, deflating Cholesky
                           normalisation; the learned correction, when
                           enabled, follows block-OSRC as in the per-rhs
                           cycle); restart then counts block steps of nrhs
                           vectors.  0: one Krylov space per right-hand
                           side.  Default 1                                  */
  int32_t mv_tensor;    /* mixed mode: 1: applies to more than 4 right-hand
                           sides at once run on the tensor cores: the FP32
                           matvec of the inner solver (mtf_matvec_f32) from
                           an FP16 hi + lo split of the stored blocks (about
                           22 significant bits, FP32 accumulation), reading
                           every stored entry once for up to 32 right-hand
                           sides, and the FP16 block-OSRC apply; applies to
                           at most 4 (one pass of the FMA streams, which are
                           faster there) and mv_tensor = 0 use the FMA
                           streams, one pass per 4.  Default 1               */
  int32_t residual_fp64;/* mixed mode: 1: the assembly also forms the FP64
                           blocks (FP64 regular and singular pairs, kept as
                           FP64 and as FP32 pairs, 64 B per entry more) and
                           the outer refinement residuals b - M x apply them
                           with double-float sums (about 2^-46), so the solution
                           converges to the FP64-assembled system's rather
                           than to the FP32-stored one's (whose difference
                           is the FP32 entry error, about 1e-7, times the
                           conditioning); mtf_matvec then applies the FP64
                           blocks.  0: residuals of the FP32-stored blocks
                           (residual_df).  Default 0                         */
  double inner_tol_min; /* mixed mode: lower bound of the relative tolerance
                           given to an inner FP32 FGMRES cycle (the cycle's
                           target is 0.3 tol / (current FP64 residual),
                           clamped to [inner_tol_min, 0.5]); a smaller bound
                           lets the first cycle run further before the FP64
                           residual is taken, a larger one restarts sooner.
                           0 selects the default 1e-5; otherwise in
                           [1e-9, 0.5]                                       */
  int32_t gs_dots_half; /* mixed mode, block_krylov with mv_tensor: 1: the
                           Gram-Schmidt dots V^H W read the FP16 high part of
                           the stored basis only (two tensor-core products
                           instead of three, half the basis bytes); the
                           second Gram-Schmidt pass measures what the first
                           left, and the update W -= V H keeps hi + lo.
                           0: hi + lo.  Default 1                            */
  int32_t osrc_type;    /* block-OSRC variant (Sec. 5.4 names Type 1 and Type
                           2; the paper defines neither beyond Eq. 19):
                           1: T~ = W diag(f) W^T with the Pade symbols f;
                           2: the compressed T~2 = W diag(f2) W^T, f2 = the
                           modulus of f with the phase of the EtM principal
                           symbol (-i |f| on irrotational, +i |f| on loop and
                           harmonic modes), so T~2 = i R with R real
                           symmetric; the wide tensor-core applies (more than
                           4 right-hand sides, mixed mode) stream R in FP16,
                           2 bytes per entry instead of 4.  The solution does
                           not depend on the choice.  0 selects 1.  Default 1 */
} mtf_options;

typedef struct {
  int32_t iterations;   /* inner (F)GMRES iterations, max over right-hand sides */
  int32_t restarts;     /* restart cycles of the slowest right-hand side        */
  int32_t refinements;  /* outer refinement steps (mixed precision)             */
  int32_t converged;    /* 1 if every right-hand side met tol                   */
  double rel_residual;  /* max over rhs of the final true ||b - M x|| / ||b||  */
  double seconds;       /* wall time of the call                               */
  double launch_seconds;/* host time spent queueing the kernels of the inner
                           block FGMRES steps (0 for other paths)            */
  double lsq_seconds;   /* host time of their block least-squares updates    */
  double wait_seconds;  /* host time spent waiting for their steps to finish
                           on the device (small when the host is the
                           bottleneck)                                       */
} mtf_solve_stats;

/* Fill *opt with the defaults listed above.  Never fails. */
void mtf_default_options(mtf_options* opt);

/* Skeleton mesh and subdomain spaces (Sec. 3.2, Sec. 4.2, Algorithm 1).
 *   vertices: nv * 3 doubles (host).
 *   tris:     nt * 3 int32 vertex ids (host); the right-hand-rule normal of
 *             triangle t points from subdomain labels[2t] into labels[2t+1].
 *   labels:   nt * 2 int32 (host), distinct, in [0, n_domains); 0 = exterior.
 *             Triangles with labels[2t] > labels[2t+1] are re-oriented so
 *             every interface Gamma_ij has its normal from min(i,j) to
 *             max(i,j), the convention Algorithm 1 assumes.
 *   n_domains: M + 1.
 * Algorithm 1 then gives, per subdomain i, the triangles of Gamma_i with
 * swap = sign(j - i) and the RWG dofs of Gamma_i.  Fails with MTF_ERR_MESH
 * unless every Gamma_i is a closed surface (each of its edges on exactly two
 * of its triangles) and every subdomain has at least one triangle.
 * Host-only: the mesh tables are uploaded to the current CUDA device by the
 * first mtf_assemble that uses the mesh (so this call, mtf_mesh_info and
 * mtf_mesh_pair_counts work without a GPU).  */
mtf_status mtf_mesh_create(const double* vertices, int32_t nv, const int32_t* tris, int32_t nt,
                           const int32_t* labels, int32_t n_domains, mtf_mesh* out);

/* n_dofs (host, n_domains entries) receives N_i = dim RWG_i; n_total
 * receives N = 2 sum N_i (Eq. 16).  Either pointer may be NULL. */
mtf_status mtf_mesh_info(mtf_mesh mesh, int32_t* n_dofs, int64_t* n_total);

/* Number of singular triangle pairs of each kind summed over blocks
 * (coincident, common edge, common vertex) and of regular pairs. */
mtf_status mtf_mesh_pair_counts(mtf_mesh mesh, int64_t* counts4);

void mtf_mesh_destroy(mtf_mesh mesh);

/* Galerkin assembly of the MTF operator M = 2A + X of Problem 2.
 *   k0:    exterior wavenumber (> 0).
 *   eps_r, mu_r: n_domains doubles each (host), relative permittivity and
 *          permeability; k_i = k0 sqrt(eps_r mu_r), rho_i = sqrt(eps_r / mu_r)
 *          (Eq. 1).  Index 0 is the exterior.
 *   opt:   NULL = defaults.
 * Builds, per block i, the dense EFIO T_i and MFIO K_i Galerkin matrices
 * at k_i (Eqs. 7-9) tested with the x-pairing (Eq. 5) -- regular pairs with
 * the 6x6-point tensor rule, coincident / common-edge / common-vertex pairs
 * with Sauter-Schwab rules -- and the sparse transmission Grams of Eq. (18)
 * for the exchange X (Eqs. 11-13).  All data stays on the device. */
mtf_status mtf_assemble(mtf_mesh mesh, double k0, const double* eps_r, const double* mu_r,
                        const mtf_options* opt, void* stream, mtf_system* out);

/* Assemble again into an existing system (same mesh and options, new k0 /
 * materials), reusing its device buffers; same definitions as mtf_assemble. */
mtf_status mtf_reassemble(mtf_system sys, double k0, const double* eps_r, const double* mu_r,
                          void* stream);

/* Kernel accounting (no counterpart in the paper; used to measure the
 * library).  Launch counts of every library kernel are always kept; with
 * mtf_profile_enable(1) each launch is also bracketed by CUDA events on its
 * stream.  mtf_profile_read(n, launches, ms) synchronises on the recorded
 * events, writes for kernel ids 0..n-1 the launches and device milliseconds
 * accumulated since the previous read (either array may be NULL) and resets
 * the counters.  Process-wide, not thread-safe. */
mtf_status mtf_profile_enable(int32_t on);
mtf_status mtf_profile_read(int32_t n, int64_t* launches, double* ms);
/* mtf_profile_read that also returns, per kernel id, the algorithmic bytes
 * of the launches counted (every stored operator entry, input and output
 * value once, as the launch site declares them; 0 for kernels that declare
 * none).  Resets all three counters. */
mtf_status mtf_profile_read_bytes(int32_t n, int64_t* launches, double* ms, double* bytes);
int32_t mtf_kernel_count(void);
const char* mtf_kernel_name(int32_t id);

/* Copy T_i and K_i (N_i x N_i complex128 each, row-major, row = test dof,
 * column = trial dof) into device buffers t_out / k_out. */
mtf_status mtf_get_block(mtf_system sys, int32_t i, void* t_out, void* k_out, void* stream);

/* y = M x (Problem 2): block-dense 2 A_i u_i plus the skeleton exchange
 * sum_j G^{ij} u_j in both trace slots (Remark 2).  x, y: device complex128,
 * n_total x nrhs, must not overlap.  Mixed-precision systems apply their
 * FP32-stored blocks with double-float sums (opt.residual_df, default) or
 * FP64 sums: the refinement residual. */
mtf_status mtf_matvec(mtf_system sys, const void* x, void* y, int32_t nrhs, void* stream);

/* z = A~ r: the block-OSRC preconditioner of Sec. 4.4 (Eq. 19),
 * A~_i = [[0, rho_i^-1 T~], [-rho_i T~, 0]] per block, with T~ the Pade
 * OSRC approximation of the EtM map (order opt.osrc_np, branch-cut angle
 * opt.osrc_theta, damped wavenumber k_i + i eps_i) evaluated on the
 * spectral decomposition of the block's RWG div-div / mass pencil.  Maps
 * tested residual vectors to coefficient vectors.  r, z: device complex128
 * n_total x nrhs, must not overlap.  Requires opt.precond == MTF_PRECOND_OSRC
 * at assembly (MTF_ERR_ARG otherwise). */
mtf_status mtf_precond_apply(mtf_system sys, const void* r, void* z, int32_t nrhs, void* stream);

/* y = M x (Eq. 16) with complex64 vectors: the FP32 streaming matvec run by
 * the mixed-precision inner solver (FP32 products and sums over the FP32-
 * stored blocks, the exchange rows X x in FP64, the result rounded to FP32).
 * Requires opt.precision == MTF_PREC_MIXED at assembly (MTF_ERR_ARG
 * otherwise).  x, y: device complex64 n_total x nrhs, must not overlap.
 * Synchronises `stream`; MTF_ERR_TIMEOUT if a bulk copy of the kernel did
 * not complete within its time limit (the output is then undefined). */
mtf_status mtf_matvec_f32(mtf_system sys, const void* x, void* y, int32_t nrhs, void* stream);

/* y = M^H v with complex64 vectors (mixed precision): the conjugate
 * transpose of mtf_matvec_f32, evaluated with T_i and K_i taken as complex
 * symmetric (their Galerkin forms are, and the assembly keeps them so to
 * rounding: both orderings of a triangle pair come from one rule) and the
 * real symmetric exchange matrix.  Used for gradients of the learned correction.  Synchronises
 * `stream`; MTF_ERR_TIMEOUT as mtf_matvec_f32. */
mtf_status mtf_matvec_adjoint_f32(mtf_system sys, const void* v, void* y, int32_t nrhs, void* stream);

/* z = A~ r (Eq. 19) with complex64 vectors: the FP32 apply the mixed inner
 * solver runs.  Same operator and requirements as mtf_precond_apply; r, z:
 * device complex64 n_total x nrhs, must not overlap. */
mtf_status mtf_precond_apply_f32(mtf_system sys, const void* r, void* z, int32_t nrhs, void* stream);

/* Right-hand side of Problem 2 for plane waves E_inc = p exp(i k0 d.x)
 * (Eq. 22): block 0 holds -2 <gamma_{.,0} E_inc, psi_m>_x for the D and N
 * slots (sign from the Calderon identities of Eq. 10 with n_0), all other
 * blocks are zero.  dirs: nrhs * 3 doubles (host, unit); pols: nrhs * 3
 * complex128 (host, orthogonal to d); b_out: device complex128 n_total x nrhs. */
mtf_status mtf_rhs(mtf_system sys, int32_t nrhs, const double* dirs, const double* pols,
                   void* b_out, void* stream);

/* Solve M u = b for nrhs plane waves with restarted flexible GMRES
 * (Sec. 5.3: relative tolerance, iteration cap), right-preconditioned by
 * block-OSRC when opt.precond says so.  x_out: device complex128
 * n_total x nrhs.  stats: host, may be NULL.  Returns MTF_ERR_NOCONV (with
 * x_out holding the last iterate) if some right-hand side misses tol. */
mtf_status mtf_solve(mtf_system sys, int32_t nrhs, const double* dirs, const double* pols,
                     void* x_out, mtf_solve_stats* stats, void* stream);

/* Solve M u = b (Problem 2) for nrhs given right-hand sides with the solver
 * of mtf_solve (same options, preconditioning, refinement and stopping test
 * relative to ||b|| per right-hand side).  b: device complex128
 * n_total x nrhs (read only); x_out: device complex128 n_total x nrhs, must
 * not overlap b.  Used e.g. for refinement against another system's
 * residuals.  Errors as mtf_solve. */
mtf_status mtf_solve_rhs(mtf_system sys, int32_t nrhs, const void* b, void* x_out, mtf_solve_stats* stats,
                         void* stream);

/* mtf_solve without device allocation (the paper has no counterpart; this
 * is an interface for callers that cannot allocate).  Some callers must not
 * call cudaMalloc while they run: code working inside a fixed, pre-reserved
 * memory budget that a late allocation could exhaust, or a serving loop /
 * host callback where cudaMalloc may implicitly synchronise the device and
 * stall other work.  This entry point runs the algorithm of mtf_solve's FP64
 * path -- restarted flexible GMRES, right-preconditioned by block-OSRC when
 * the system was assembled with MTF_PRECOND_OSRC, CGS2 orthogonalisation,
 * Givens rotations on the host -- with its own simpler reduction kernels, so
 * its results agree with mtf_solve to rounding (1e-10 relative), not bit for
 * bit.  It takes every device buffer it needs -- right-hand sides, Krylov
 * basis, preconditioned directions, work vectors, Hessenberg columns, wave
 * parameters -- from one static device array of 16 MiB that every GPU
 * loading the library holds until the process exits (block-OSRC systems
 * prepare their apply tables at assembly).  The caller still provides x_out.
 *   Limit, in doubles, with n = n_total and m = opt.restart:
 *     2 n nrhs (m + 4) + (6 m + 8) nrhs + 9 nrhs + 64
 *   plus 2 n nrhs m + n nrhs with block-OSRC, must fit in 2^21; larger
 *   requests fail with MTF_ERR_ARG and a message giving both numbers.
 *   Set-up: the first call on each device (with that device current) looks
 *   up the array's device address; make that first call before any stream
 *   capture.
 *   Sharing: every call on a device uses the same array and leaves its
 *   contents behind (each call clears the part it uses first).  Calls whose
 *   GPU work overlaps -- on different streams or from different threads --
 *   race on the array and give wrong results; serialise them.
 * Only systems assembled with MTF_PREC_FP64 are accepted (MTF_ERR_ARG
 * otherwise).  Arguments, results and errors are those of mtf_solve. */
mtf_status mtf_solve_static(mtf_system sys, int32_t nrhs, const double* dirs, const double* pols,
                            void* x_out, mtf_solve_stats* stats, void* stream);

/* Batched solve of independent problems: each instance is Problem 2 on its
 * own system, solved as mtf_solve solves it (Sec. 5.3 stopping rule per
 * right-hand side).  The paper solves one scatterer at a time; the batch is
 * this library's, for workloads of many small, uneven instances whose single
 * solves leave most of the GPU idle (their kernels are short and their
 * steps wait on each other).  Instance i solves the nrhs[i] plane waves
 * dirs[i], pols[i] (host, laid out as for mtf_solve) on systems[i] into
 * x_out[i] (device complex128 n_total_i x nrhs[i]).  The instances run
 * concurrently: each on its own CUDA stream, driven by a pool of host worker
 * threads (at most `threads`; threads <= 0 selects min(n, 4), the best of
 * 4 to 32 measured on 32 uneven instances), largest
 * instance (n_total x nrhs) first.  They start after the work queued on
 * `stream` before the call, and the call returns when every instance has
 * finished.  systems: n distinct handles, all on the current device (a
 * system must not be used by two calls at once).  stats: host array of n
 * entries, may be NULL.  Returns MTF_OK, or the status of the
 * lowest-indexed failing instance (every instance runs to its end);
 * MTF_ERR_ARG for n < 1, null arrays or a repeated system. */
mtf_status mtf_solve_batch(int32_t n, const mtf_system* systems, const int32_t* nrhs, const double* const* dirs,
                           const double* const* pols, void* const* x_out, mtf_solve_stats* stats, int32_t threads,
                           void* stream);

/* Arithmetic-peak probes of the current device (a measurement utility of
 * this library; no counterpart in the paper): rates[0] = FP32 FLOP/s (fused
 * multiply-add chains, an FMA counts 2), rates[1] = FP64 FLOP/s, rates[2] =
 * special-function results per second (single-precision sine on the SFU).
 * Independent chains per thread over 8 CTAs of 256 threads per SM, timed
 * with CUDA events on `stream` after one warm-up launch; about 2 ms.
 * rates: host, 3 doubles. */
mtf_status mtf_probe_peaks(double* rates, void* stream);

/* Autotuner of the mixed inner solver's operator applies (this library's;
 * no counterpart in the paper).  For nrhs right-hand sides per apply it times
 * the candidate launch plans of mtf_matvec_f32 on the system -- the FMA
 * stream (one pass per 4 right-hand sides) and the tensor-core kernel with
 * work units of {2, 8}-chunk minimum pieces at {2, 4, 8} units per CTA on
 * all SMs or half of them -- with CUDA events on `stream` (one warm-up and
 * `reps` timed applies each, on a fixed input), and keeps the fastest for
 * every later apply of the system (matvec and block-OSRC, which share the
 * plan).  Applies to at most 4 right-hand sides always use the FMA stream,
 * so for nrhs <= 4 only that candidate exists.  report: host, may be NULL:
 * one line per candidate ("<plan> <mean ms>") and a last line "chosen
 * <plan>", NUL-terminated within report_len bytes.  Mixed-precision systems
 * with mv_tensor only (MTF_ERR_ARG otherwise); reps in 1..100. */
mtf_status mtf_autotune(mtf_system sys, int32_t nrhs, int32_t reps, char* report, int32_t report_len, void* stream);

/* ---------------------------------------------------------------------------
 * Learned correction of the block-OSRC preconditioner (no counterpart in the
 * paper).  The preconditioner stays linear: z = P r + C r, P the block-OSRC
 * operator of Eq. 19 and C a local stencil.  For dof m of block i and its 4
 * RWG neighbours (the other edges of its two triangles on Gamma_i, ascending
 * local dof index) -- stencil slots q = 0 (m) .. 4 -- and sources s in
 * {r, P r}:
 *   (C r)_D[m] = sum_{q,s} a[q,s,DD] s_D[q] + a[q,s,DN] s_N[q]
 *   (C r)_N[m] = sum_{q,s} a[q,s,ND] s_D[q] + a[q,s,NN] s_N[q],
 * 80 reals per dof, the (re, im) of a ordered [q][s][DD, DN, ND, NN].
 * Parametrisations (mtf_learned_kind):
 *  - MTF_LEARNED_TABLE: the coefficients are the parameters, float
 *    80 x n_dofs feature-major (coefficient o of dof row g at [o n_dofs + g]);
 *  - MTF_LEARNED_NETWORK: a = g(x) per dof, g a network of 10 geometric
 *    features (k_i l_m, rho_i, 1 for block 0, k_i l of the 4 neighbours,
 *    k_i^2 (A_1 + A_2) of its triangles, cosine between their normals, 1 for
 *    a junction edge) -> 256 -> 256 (ReLU) -> 80; parameters augmented
 *    row-major matrices [W | b] layer after layer (256 x 11, 256 x 257,
 *    80 x 257); every layer's product (forward, backward, weight gradient)
 *    runs on the tensor cores (FP16 hi + lo operands, FP32 accumulation).
 * Both start at zero output (plain block-OSRC).  Training minimises the
 * power loss
 *   L = mean_z ||E^K z||^2 / ||z||^2,   E = I - M (P + C) / c0,
 * over complex Rademacher vectors z, c0 the mean Rayleigh quotient
 * <z, M P z> / <z, z> of the plain preconditioned operator: a stochastic
 * estimate of sum_i |1 - lambda_i / c0|^(2K) over the eigenvalues of
 * M (P + C), dominated by the outliers that slow restarted GMRES.  Inside
 * flexible GMRES the correction changes only the iteration count.  Rows are
 * the global dof rows, n_dofs = n_total / 2.  All entry points need a system
 * assembled with MTF_PRECOND_OSRC (training: also MTF_PREC_MIXED); device
 * arrays must not overlap.
 * ------------------------------------------------------------------------- */
typedef enum {
  MTF_LEARNED_TABLE = 0,
  MTF_LEARNED_NETWORK = 1
} mtf_learned_kind;

/* Number of float parameters (0 before mtf_learned_init). */
int64_t mtf_learned_param_count(mtf_system sys);

/* Create the correction: `kind` (mtf_learned_kind); the network's hidden
 * layers He-uniform from `seed`, every output zero; resets Adam. */
mtf_status mtf_learned_init(mtf_system sys, int32_t kind, uint64_t seed);

/* Copy the parameters to / from host memory (mtf_learned_param_count floats). */
mtf_status mtf_learned_get_params(mtf_system sys, float* host_params);
mtf_status mtf_learned_set_params(mtf_system sys, const float* host_params);

/* Geometric features of every dof: x_out device float 10 x n_dofs,
 * feature-major.  Synchronises `stream`. */
mtf_status mtf_learned_features(mtf_system sys, void* x_out, void* stream);

/* Network only: loss sum_q w_q |g(x_q) - t_q|^2 and its gradient; x device
 * float 10 x rows, t device float 80 x rows (feature-major, leading
 * dimension rows), w device float rows; grad_out device float (param
 * count); *loss on host.  Synchronises `stream`. */
mtf_status mtf_learned_loss_grad(mtf_system sys, const void* x, const void* t, const void* w, int64_t rows,
                                 void* grad_out, double* loss, void* stream);

/* Power loss of K steps (1..16) on given vectors z (device complex64
 * n_total x ncols, ncols <= 32) with centre c0 = c0_re + i c0_im, and its
 * gradient with respect to the parameters (grad_out device float, param
 * count); *loss on host.  Synchronises `stream`. */
mtf_status mtf_learned_power_grad(mtf_system sys, const void* z, int32_t ncols, double c0_re, double c0_im,
                                  int32_t K, void* grad_out, double* loss, void* stream);

/* Adjoint of the stencil: out_r = C_r^H w and out_p = C_P^H w, with C r =
 * C_r r + C_P (P r); w, out_r, out_p device complex64 n_total x nrhs. */
mtf_status mtf_learned_stencil_adjoint(mtf_system sys, const void* w, void* out_r, void* out_p, int32_t nrhs,
                                       void* stream);

/* Adjoint of block-OSRC: z = P^H w (complex64 device n_total x nrhs). */
mtf_status mtf_precond_adjoint_f32(mtf_system sys, const void* w, void* z, int32_t nrhs, void* stream);

/* Centre c0 of the power loss (real part returned, imaginary part in *im if
 * not NULL), estimated over 64 random vectors on first use. */
double mtf_learned_centre(mtf_system sys, double* im);

/* `steps` Adam steps (learning rate lr) of the power loss with K steps on
 * `batch` (<= 32) fresh random vectors each, drawn from `seed`; the loss of
 * the first and of the last step on host.  Synchronises `stream`. */
mtf_status mtf_learned_train(mtf_system sys, int32_t steps, double lr, int32_t batch, int32_t K, uint64_t seed,
                             double* loss_first, double* loss_last, void* stream);

typedef struct {
  int32_t plain_iterations;  /* validation solve with plain block-OSRC        */
  int32_t best_iterations;   /* best validation solve (plain if not improved) */
  int32_t best_round;        /* round of the kept parameters, 0 = none        */
  int32_t rounds;            /* training rounds run                           */
  double loss_first;         /* power loss of the first training step         */
  double loss_last;          /* power loss of the last training step          */
  int32_t enabled;           /* 1 if the correction is switched on            */
} mtf_learned_report;

/* Train in `rounds` rounds of steps_per_round mtf_learned_train steps and,
 * after each, solve the n_val plane waves (host dirs / pols as in mtf_rhs)
 * with the correction; keep the parameters of the round with the fewest
 * iterations and switch the correction on if that beats plain block-OSRC,
 * else switch it off.  Needs a mixed-precision system.  Synchronises
 * `stream`. */
mtf_status mtf_learned_fit(mtf_system sys, int32_t n_val, const double* dirs, const double* pols, int32_t rounds,
                           int32_t steps_per_round, double lr, int32_t batch, int32_t K, uint64_t seed,
                           mtf_learned_report* report, void* stream);

/* Switch the correction on (1) or off (0) for later mtf_solve calls of this
 * system (the assembly option `learned` sets the initial state). */
mtf_status mtf_learned_enable(mtf_system sys, int32_t on);

/* z = P r + C r for nrhs columns, complex64 device n_total x nrhs. */
mtf_status mtf_learned_apply(mtf_system sys, const void* r, void* z, int32_t nrhs, void* stream);

/* Far field E_inf(xhat) of solutions x (device complex128 n_total x nrhs) at
 * n_obs unit directions obs_dirs (host, n_obs * 3 doubles):
 * E_inf = i k0 / (4 pi) [xhat x w_D + (xhat x w_N) x xhat],
 * w_. = int_{Gamma_0} (trace) exp(-i k0 xhat . y) dy, from the Stratton-Chu
 * representation (Eq. 8) in Omega_0 (RCS_z of Sec. 5.2 is its z component).
 * f_out: device complex128, n_obs * 3 * nrhs, index (c * n_obs + o) * 3 + xyz. */
mtf_status mtf_farfield(mtf_system sys, const void* x, int32_t nrhs, const double* obs_dirs,
                        int32_t n_obs, void* f_out, void* stream);

/* Near field by the representation formula (Eq. 8): for every point x_p
 * (host, n_pts * 3 doubles) in subdomain domains[p] (host int32, 0..M),
 *   U(x_p) = H_{k_i}(gamma_D U) + E_{k_i}(gamma_N U)
 * from block i = domains[p] of the solutions x (device complex128
 * n_total x nrhs): the scattered field in Omega_0, the total field in
 * Omega_i (i >= 1).  6-point rule per triangle: points should keep about one
 * triangle diameter from the skeleton.  f_out: device complex128,
 * n_pts * 3 * nrhs, index (c * n_pts + p) * 3 + xyz.  Synchronises `stream`. */
mtf_status mtf_nearfield(mtf_system sys, const void* x, int32_t nrhs, const double* points, const int32_t* domains,
                         int32_t n_pts, void* f_out, void* stream);

void mtf_system_destroy(mtf_system sys);

const char* mtf_status_string(mtf_status s);
const char* mtf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MTF_H_ */
