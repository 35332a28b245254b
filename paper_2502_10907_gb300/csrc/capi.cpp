// C-ABI of libmtf (declared in include/mtf.h).  Every entry point converts
// internal errors into an mtf_status and records a message for
// mtf_last_error(); nothing throws across the boundary.
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include <algorithm>
#include <atomic>

#include "common.h"

namespace mtf {
mtf_mesh build_mesh(const double* V, int32_t nv, const int32_t* F, int32_t nt, const int32_t* L, int32_t nd);
void upload_mesh(mtf_mesh m, cudaStream_t s);

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

template <class Fn>
static mtf_status guarded(Fn&& fn) {
  try {
    fn();
    return MTF_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return MTF_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return MTF_ERR_ARG;
  }
}

static void upload_small(DevBuf<double>& buf, const double* h, size_t n, cudaStream_t s) {
  if (buf.n < n) buf.alloc(n);
  MTF_CUDA(cudaMemcpyAsync(buf.p, h, n * sizeof(double), cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaStreamSynchronize(s));
}
}  // namespace mtf

namespace mtf {
void assemble_into(mtf_system sys, double k0, const double* eps_r, const double* mu_r, cudaStream_t s) {
  mtf_mesh mesh = sys->mesh;
  sys->k0 = k0;
  std::vector<double> kk(2 * mesh->nd), rr(2 * mesh->nd);
  sys->k_re.clear();
  sys->k_im.clear();
  sys->rho_re.clear();
  sys->rho_im.clear();
  for (int i = 0; i < mesh->nd; ++i) {
    MTF_REQUIRE(eps_r[i] > 0 && mu_r[i] > 0 && std::isfinite(eps_r[i]) && std::isfinite(mu_r[i]), MTF_ERR_ARG,
                "eps_r and mu_r must be positive");
    // k_i = k0 sqrt(eps mu), rho_i = sqrt(eps / mu)  (Eq. 1)
    const double ki = k0 * std::sqrt(eps_r[i] * mu_r[i]);
    const double ri = std::sqrt(eps_r[i] / mu_r[i]);
    kk[2 * i] = ki;
    kk[2 * i + 1] = 0.0;
    rr[2 * i] = ri;
    rr[2 * i + 1] = 0.0;
    sys->k_re.push_back(ki);
    sys->k_im.push_back(0.0);
    sys->rho_re.push_back(ri);
    sys->rho_im.push_back(0.0);
  }
  upload_small(sys->d_k, kk.data(), kk.size(), s);
  upload_small(sys->d_rho, rr.data(), rr.size(), s);
  // FP32 (rho, 1 / rho) per block for the FP32 epilogues
  std::vector<float> r32(4 * mesh->nd);
  for (int i = 0; i < mesh->nd; ++i) {
    const std::complex<double> r(rr[2 * i], rr[2 * i + 1]), ri = 1.0 / r;
    r32[4 * i] = float(r.real());
    r32[4 * i + 1] = float(r.imag());
    r32[4 * i + 2] = float(ri.real());
    r32[4 * i + 3] = float(ri.imag());
  }
  sys->d_rho32.alloc(r32.size());
  MTF_CUDA(cudaMemcpyAsync(sys->d_rho32.p, r32.data(), r32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  MTF_CUDA(cudaStreamSynchronize(s));
  launch_assemble(sys, s);
  if (sys->opt.precond == MTF_PRECOND_OSRC) osrc_setup(sys, s);
}
}  // namespace mtf

using namespace mtf;

extern "C" {

void mtf_default_options(mtf_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MTF_PREC_FP64;
  o->n_ss = 4;
  o->restart = 100;
  o->max_iter = 2000;
  o->tol = 1e-5;
  o->precond = MTF_PRECOND_NONE;
  o->osrc_np = 4;
  o->osrc_theta = M_PI / 2;
  o->osrc_eps_scale = 0.39;
  o->max_refine = 4;
  o->osrc_half = 1;
  o->recycle = 1;
  o->residual_df = 1;
  o->block_krylov = 1;
  o->mv_tensor = 1;
  o->gs_dots_half = 1;
  o->osrc_type = 1;
}

mtf_status mtf_mesh_create(const double* vertices, int32_t nv, const int32_t* tris, int32_t nt,
                           const int32_t* labels, int32_t n_domains, mtf_mesh* out) {
  return guarded([&] {
    MTF_REQUIRE(out, MTF_ERR_ARG, "out is null");
    *out = nullptr;
    *out = build_mesh(vertices, nv, tris, nt, labels, n_domains);
  });
}

mtf_status mtf_mesh_info(mtf_mesh mesh, int32_t* n_dofs, int64_t* n_total) {
  return guarded([&] {
    MTF_REQUIRE(mesh, MTF_ERR_ARG, "mesh is null");
    if (n_dofs)
      for (int i = 0; i < mesh->nd; ++i) n_dofs[i] = mesh->blk[i].N;
    if (n_total) *n_total = mesh->n_total;
  });
}

mtf_status mtf_mesh_pair_counts(mtf_mesh mesh, int64_t* counts4) {
  return guarded([&] {
    MTF_REQUIRE(mesh && counts4, MTF_ERR_ARG, "null argument");
    for (int c = 0; c < 4; ++c) counts4[c] = mesh->pair_counts[c];
  });
}

void mtf_mesh_destroy(mtf_mesh mesh) { delete mesh; }

mtf_status mtf_assemble(mtf_mesh mesh, double k0, const double* eps_r, const double* mu_r,
                        const mtf_options* opt, void* stream, mtf_system* out) {
  return guarded([&] {
    MTF_REQUIRE(mesh && eps_r && mu_r && out, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(k0 > 0 && std::isfinite(k0), MTF_ERR_ARG, "k0 must be positive");
    *out = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto* sys = new mtf_system_s();
    try {
      sys->mesh = mesh;
      if (!mesh->uploaded) {
        upload_mesh(mesh, s);
        mesh->uploaded = true;
      }
      if (opt) sys->opt = *opt;
      else mtf_default_options(&sys->opt);
      MTF_REQUIRE(sys->opt.n_ss >= 1 && sys->opt.n_ss <= 12, MTF_ERR_ARG, "n_ss out of range 1..12");
      MTF_REQUIRE(sys->opt.precision == MTF_PREC_FP64 || sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG,
                  "unknown precision");
      MTF_REQUIRE(sys->opt.precond == MTF_PRECOND_NONE || sys->opt.precond == MTF_PRECOND_OSRC, MTF_ERR_ARG,
                  "unknown preconditioner");
      MTF_REQUIRE(sys->opt.osrc_half == 0 || sys->opt.osrc_half == 1, MTF_ERR_ARG, "osrc_half must be 0 or 1");
      MTF_REQUIRE(sys->opt.recycle == 0 || sys->opt.recycle == 1, MTF_ERR_ARG, "recycle must be 0 or 1");
      MTF_REQUIRE(sys->opt.residual_df == 0 || sys->opt.residual_df == 1, MTF_ERR_ARG,
                  "residual_df must be 0 or 1");
      MTF_REQUIRE(sys->opt.block_krylov == 0 || sys->opt.block_krylov == 1, MTF_ERR_ARG,
                  "block_krylov must be 0 or 1");
      MTF_REQUIRE(sys->opt.mv_tensor == 0 || sys->opt.mv_tensor == 1, MTF_ERR_ARG, "mv_tensor must be 0 or 1");
      MTF_REQUIRE(sys->opt.residual_fp64 == 0 || sys->opt.residual_fp64 == 1, MTF_ERR_ARG,
                  "residual_fp64 must be 0 or 1");
      MTF_REQUIRE(sys->opt.inner_tol_min == 0.0 || (sys->opt.inner_tol_min >= 1e-9 && sys->opt.inner_tol_min <= 0.5),
                  MTF_ERR_ARG, "inner_tol_min must be 0 or in [1e-9, 0.5]");
      MTF_REQUIRE(sys->opt.gs_dots_half == 0 || sys->opt.gs_dots_half == 1, MTF_ERR_ARG,
                  "gs_dots_half must be 0 or 1");
      if (sys->opt.osrc_type == 0) sys->opt.osrc_type = 1;
      MTF_REQUIRE(sys->opt.osrc_type == 1 || sys->opt.osrc_type == 2, MTF_ERR_ARG, "osrc_type must be 1 or 2");
      MTF_REQUIRE(sys->opt.osrc_np >= 1 && sys->opt.osrc_np <= 16, MTF_ERR_ARG, "osrc_np out of range 1..16");
      assemble_into(sys, k0, eps_r, mu_r, s);
    } catch (...) {
      delete sys;
      throw;
    }
    *out = sys;
  });
}

mtf_status mtf_reassemble(mtf_system sys, double k0, const double* eps_r, const double* mu_r, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && eps_r && mu_r, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(k0 > 0 && std::isfinite(k0), MTF_ERR_ARG, "k0 must be positive");
    assemble_into(sys, k0, eps_r, mu_r, static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_profile_enable(int32_t on) {
  return guarded([&] { prof_enable(on != 0); });
}

mtf_status mtf_profile_read(int32_t n, int64_t* launches, double* ms) {
  return guarded([&] {
    MTF_REQUIRE(n >= 0, MTF_ERR_ARG, "n must be >= 0");
    prof_read(n, launches, ms);
  });
}

mtf_status mtf_profile_read_bytes(int32_t n, int64_t* launches, double* ms, double* bytes) {
  return guarded([&] {
    MTF_REQUIRE(n >= 0, MTF_ERR_ARG, "n must be >= 0");
    prof_read(n, launches, ms, bytes);
  });
}

int32_t mtf_kernel_count(void) { return KID_COUNT; }

const char* mtf_kernel_name(int32_t id) { return kernel_name(id); }

mtf_status mtf_get_block(mtf_system sys, int32_t i, void* t_out, void* k_out, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && t_out && k_out, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(i >= 0 && i < sys->mesh->nd, MTF_ERR_ARG, "block index out of range");
    launch_get_block(sys, i, static_cast<double*>(t_out), static_cast<double*>(k_out),
                     static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_matvec(mtf_system sys, const void* x, void* y, int32_t nrhs, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && x && y, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    MTF_REQUIRE(x != y, MTF_ERR_ARG, "x and y must not overlap");
    const int64_t n = sys->mesh->n_total;
    launch_matvec(sys, static_cast<const double*>(x), n, static_cast<double*>(y), n, nrhs,
                  static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_precond_apply(mtf_system sys, const void* r, void* z, int32_t nrhs, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && r && z, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    MTF_REQUIRE(r != z, MTF_ERR_ARG, "r and z must not overlap");
    MTF_REQUIRE(sys->opt.precond == MTF_PRECOND_OSRC, MTF_ERR_ARG,
                "the system was assembled without the OSRC preconditioner");
    const int64_t n = sys->mesh->n_total;
    launch_osrc_apply(sys, static_cast<const double*>(r), n, static_cast<double*>(z), n, nrhs,
                      static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_matvec_f32(mtf_system sys, const void* x, void* y, int32_t nrhs, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && x && y, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    MTF_REQUIRE(x != y, MTF_ERR_ARG, "x and y must not overlap");
    MTF_REQUIRE(sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG,
                "the FP32 matvec needs a system assembled in mixed precision");
    const int64_t n = sys->mesh->n_total;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_matvec_f32(sys, static_cast<const float*>(x), n, static_cast<float*>(y), n, nrhs, s);
    check_matvec_stream(sys, s);
  });
}

mtf_status mtf_matvec_adjoint_f32(mtf_system sys, const void* v, void* y, int32_t nrhs, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && v && y, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    MTF_REQUIRE(v != y, MTF_ERR_ARG, "v and y must not overlap");
    MTF_REQUIRE(sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG,
                "the FP32 adjoint matvec needs a system assembled in mixed precision");
    const int64_t n = sys->mesh->n_total;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_matvec_adj_f32(sys, static_cast<const float*>(v), n, static_cast<float*>(y), n, nrhs, s);
    check_matvec_stream(sys, s);
  });
}

mtf_status mtf_precond_apply_f32(mtf_system sys, const void* r, void* z, int32_t nrhs, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && r && z, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    MTF_REQUIRE(r != z, MTF_ERR_ARG, "r and z must not overlap");
    MTF_REQUIRE(sys->opt.precond == MTF_PRECOND_OSRC, MTF_ERR_ARG,
                "the system was assembled without the OSRC preconditioner");
    const int64_t n = sys->mesh->n_total;
    launch_osrc_apply_f32(sys, static_cast<const float*>(r), n, static_cast<float*>(z), n, nrhs,
                          static_cast<cudaStream_t>(stream));
  });
}

static void upload_waves(DevBuf<double>& d_dirs, DevBuf<double>& d_pols, int32_t nrhs, const double* dirs,
                         const double* pols, cudaStream_t s) {
  MTF_REQUIRE(nrhs >= 1 && dirs && pols, MTF_ERR_ARG, "need nrhs >= 1 and wave arrays");
  for (int c = 0; c < nrhs; ++c) {
    const double* d = dirs + 3 * c;
    const double nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    MTF_REQUIRE(std::fabs(nd - 1.0) < 1e-8, MTF_ERR_ARG, "directions must be unit vectors");
  }
  upload_small(d_dirs, dirs, size_t(nrhs) * 3, s);
  upload_small(d_pols, pols, size_t(nrhs) * 6, s);
}

mtf_status mtf_rhs(mtf_system sys, int32_t nrhs, const double* dirs, const double* pols, void* b_out,
                   void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && b_out, MTF_ERR_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf<double> dd, dp;
    upload_waves(dd, dp, nrhs, dirs, pols, s);
    launch_rhs(sys, nrhs, dd.p, dp.p, static_cast<double*>(b_out), s);
    MTF_CUDA(cudaStreamSynchronize(s));
  });
}

mtf_status mtf_solve(mtf_system sys, int32_t nrhs, const double* dirs, const double* pols, void* x_out,
                     mtf_solve_stats* stats, void* stream) {
  mtf_status st = MTF_OK;
  mtf_status g = guarded([&] {
    MTF_REQUIRE(sys && x_out, MTF_ERR_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the buffers stay with the system (no allocation, and no implicit
    // device synchronisation, in repeated solves)
    upload_waves(sys->d_wdir, sys->d_wpol, nrhs, dirs, pols, s);
    const size_t nb = size_t(sys->mesh->n_total) * nrhs * 2;
    if (sys->d_brhs.n < nb) sys->d_brhs.alloc(nb);
    launch_rhs(sys, nrhs, sys->d_wdir.p, sys->d_wpol.p, sys->d_brhs.p, s);
    st = solve(sys, nrhs, sys->d_brhs.p, static_cast<double*>(x_out), stats, s);
    MTF_CUDA(cudaStreamSynchronize(s));
    if (st == MTF_ERR_NOCONV) set_last_error("GMRES did not reach the tolerance within max_iter");
    if (st == MTF_ERR_NAN) set_last_error("non-finite residual in GMRES");
  });
  return g != MTF_OK ? g : st;
}

mtf_status mtf_solve_rhs(mtf_system sys, int32_t nrhs, const void* b, void* x_out, mtf_solve_stats* stats,
                         void* stream) {
  mtf_status st = MTF_OK;
  mtf_status g = guarded([&] {
    MTF_REQUIRE(sys && b && x_out, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1, MTF_ERR_ARG, "nrhs must be >= 1");
    MTF_REQUIRE(b != x_out, MTF_ERR_ARG, "b and x_out must not overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = solve(sys, nrhs, static_cast<const double*>(b), static_cast<double*>(x_out), stats, s);
    MTF_CUDA(cudaStreamSynchronize(s));
    if (st == MTF_ERR_NOCONV) set_last_error("GMRES did not reach the tolerance within max_iter");
    if (st == MTF_ERR_NAN) set_last_error("non-finite residual in GMRES");
  });
  return g != MTF_OK ? g : st;
}

// ---------------------------------------------------------------------------
// batched solve and autotuner
// ---------------------------------------------------------------------------
mtf_status mtf_solve_batch(int32_t n, const mtf_system* systems, const int32_t* nrhs, const double* const* dirs,
                           const double* const* pols, void* const* x_out, mtf_solve_stats* stats, int32_t threads,
                           void* stream) {
  std::vector<mtf_status> status;
  std::vector<std::string> msg;
  mtf_status g = guarded([&] {
    MTF_REQUIRE(n >= 1 && systems && nrhs && dirs && pols && x_out, MTF_ERR_ARG, "batch: null arrays or n < 1");
    for (int i = 0; i < n; ++i) {
      MTF_REQUIRE(systems[i] && x_out[i] && nrhs[i] >= 1, MTF_ERR_ARG, "batch: instance " + std::to_string(i));
      for (int j = 0; j < i; ++j) MTF_REQUIRE(systems[j] != systems[i], MTF_ERR_ARG, "batch: repeated system");
    }
    int dev = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    // instances largest first, so that the long ones start early
    std::vector<int> order(static_cast<size_t>(n));
    for (int i = 0; i < n; ++i) order[size_t(i)] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return double(systems[a]->mesh->n_total) * nrhs[a] > double(systems[b]->mesh->n_total) * nrhs[b];
    });
    const int nt = std::max(1, std::min<int>(n, threads > 0 ? threads : 4));
    // every instance starts after the work queued on the caller's stream
    cudaEvent_t start = nullptr;
    MTF_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    MTF_CUDA(cudaEventRecord(start, static_cast<cudaStream_t>(stream)));
    status.assign(size_t(n), MTF_OK);
    msg.assign(size_t(n), std::string());
    std::atomic<int> next{0};
    auto worker = [&]() {
      cudaSetDevice(dev);
      cudaStream_t s = nullptr;
      if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
          status[size_t(order[size_t(q)])] = MTF_ERR_CUDA;
          msg[size_t(order[size_t(q)])] = "batch: stream creation failed";
        }
        return;
      }
      cudaStreamWaitEvent(s, start, 0);
      for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
        const int i = order[size_t(q)];
        mtf_solve_stats* st = stats ? stats + i : nullptr;
        const mtf_status r = mtf_solve(systems[i], nrhs[i], dirs[i], pols[i], x_out[i], st, s);
        status[size_t(i)] = r;
        if (r != MTF_OK) msg[size_t(i)] = mtf_last_error();
      }
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    cudaEventDestroy(start);
  });
  if (g != MTF_OK) return g;
  for (int i = 0; i < n; ++i)
    if (status[size_t(i)] != MTF_OK) {
      set_last_error("instance " + std::to_string(i) + ": " + msg[size_t(i)]);
      return status[size_t(i)];
    }
  return MTF_OK;
}

mtf_status mtf_probe_peaks(double* rates, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(rates, MTF_ERR_ARG, "null argument");
    probe_peaks(rates, static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_autotune(mtf_system sys, int32_t nrhs, int32_t reps, char* report, int32_t report_len, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && nrhs >= 1 && reps >= 1 && reps <= 100, MTF_ERR_ARG, "autotune: arguments");
    MTF_REQUIRE(tc_matvec_enabled(sys), MTF_ERR_ARG, "autotune: needs a mixed-precision system with mv_tensor");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t ldn = (sys->mesh->n_total + 63) & ~int64_t(63);  // the solvers' padded column length
    DevBuf<float> x, y;
    x.alloc(size_t(ldn) * nrhs * 2);
    y.alloc(size_t(ldn) * nrhs * 2);
    MTF_CUDA(cudaMemsetAsync(x.p, 0x3c, x.n * sizeof(float), s));  // every float 0.0115
    int dev = 0, sms = 0;
    MTF_CUDA(cudaGetDevice(&dev));
    MTF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    struct Cand {
      int waves, min_len, grid;
      bool fma;
      std::string name;
    };
    std::vector<Cand> cands{{0, 0, 0, true, "fma_stream"}};
    if (nrhs > kFmaPassRhs)
      for (int grid : {0, sms / 2})
        for (int waves : {2, 4, 8})
          for (int ml : {2, 8})
            cands.push_back({waves, ml, grid, false,
                             "tc waves=" + std::to_string(waves) + " min_len=" + std::to_string(ml) +
                                 " grid=" + std::to_string(grid > 0 ? grid : sms)});
    cudaEvent_t e0, e1;
    MTF_CUDA(cudaEventCreate(&e0));
    MTF_CUDA(cudaEventCreate(&e1));
    std::string rep;
    size_t best = 0;
    float best_ms = 0.f;
    for (size_t c = 0; c < cands.size(); ++c) {
      const Cand& k = cands[c];
      tc_set_plan(sys, k.waves, k.min_len, k.grid, k.fma, s);
      launch_matvec_f32(sys, x.p, ldn, y.p, ldn, nrhs, s);  // warm-up
      MTF_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < reps; ++r) launch_matvec_f32(sys, x.p, ldn, y.p, ldn, nrhs, s);
      MTF_CUDA(cudaEventRecord(e1, s));
      MTF_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      MTF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= float(reps);
      rep += k.name + " " + std::to_string(ms) + "\n";
      if (c == 0 || ms < best_ms) {
        best = c;
        best_ms = ms;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_matvec_stream(sys, s);
    const Cand& k = cands[best];
    tc_set_plan(sys, k.waves, k.min_len, k.grid, k.fma, s);
    rep += "chosen " + k.name + "\n";
    if (report && report_len > 0) {
      const size_t len = std::min(rep.size(), size_t(report_len - 1));
      std::memcpy(report, rep.data(), len);
      report[len] = '\0';
    }
  });
}

// ---------------------------------------------------------------------------
// learned correction of block-OSRC
// ---------------------------------------------------------------------------
int64_t mtf_learned_param_count(mtf_system sys) { return sys ? learned_param_count(sys) : 0; }

static void require_learned_system(mtf_system sys) {
  MTF_REQUIRE(sys, MTF_ERR_ARG, "null argument");
  MTF_REQUIRE(sys->opt.precond == MTF_PRECOND_OSRC, MTF_ERR_ARG,
              "the learned correction needs a system assembled with MTF_PRECOND_OSRC");
}

mtf_status mtf_learned_init(mtf_system sys, int32_t kind, uint64_t seed) {
  return guarded([&] {
    require_learned_system(sys);
    learned_init(sys, kind, seed, nullptr);
  });
}

mtf_status mtf_learned_get_params(mtf_system sys, float* host_params) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(host_params, MTF_ERR_ARG, "null argument");
    learned_get_params(sys, host_params, nullptr);
  });
}

mtf_status mtf_learned_set_params(mtf_system sys, const float* host_params) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(host_params, MTF_ERR_ARG, "null argument");
    learned_set_params(sys, host_params, nullptr);
  });
}

mtf_status mtf_learned_features(mtf_system sys, void* x_out, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(x_out, MTF_ERR_ARG, "null argument");
    learned_features(sys, static_cast<float*>(x_out), static_cast<cudaStream_t>(stream));
    MTF_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  });
}

mtf_status mtf_learned_loss_grad(mtf_system sys, const void* x, const void* t, const void* w, int64_t rows,
                                 void* grad_out, double* loss, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(x && t && w && grad_out, MTF_ERR_ARG, "null argument");
    learned_loss_grad(sys, static_cast<const float*>(x), static_cast<const float*>(t), static_cast<const float*>(w),
                      rows, static_cast<float*>(grad_out), loss, static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_learned_power_grad(mtf_system sys, const void* z, int32_t ncols, double c0_re, double c0_im, int32_t K,
                                  void* grad_out, double* loss, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(z && grad_out, MTF_ERR_ARG, "null argument");
    learned_power_grad(sys, static_cast<const float*>(z), ncols, c0_re, c0_im, K, static_cast<float*>(grad_out), loss,
                       static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_learned_stencil_adjoint(mtf_system sys, const void* w, void* out_r, void* out_p, int32_t nrhs,
                                       void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(w && out_r && out_p && nrhs >= 1, MTF_ERR_ARG, "null argument or nrhs < 1");
    learned_stencil_adjoint(sys, static_cast<const float*>(w), static_cast<float*>(out_r), static_cast<float*>(out_p),
                            nrhs, static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_precond_adjoint_f32(mtf_system sys, const void* w, void* z, int32_t nrhs, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(w && z && w != z && nrhs >= 1, MTF_ERR_ARG, "null or overlapping argument, or nrhs < 1");
    MTF_REQUIRE(sys->opt.precision == MTF_PREC_MIXED, MTF_ERR_ARG, "FP32 operators need a mixed-precision system");
    const int64_t n = sys->mesh->n_total;
    launch_osrc_apply_adj_f32(sys, static_cast<const float*>(w), n, static_cast<float*>(z), n, nrhs,
                              static_cast<cudaStream_t>(stream));
  });
}

double mtf_learned_centre(mtf_system sys, double* im) {
  double re = 1.0;
  if (im) *im = 0.0;
  guarded([&] {
    require_learned_system(sys);
    re = learned_centre(sys, im, nullptr);
  });
  return re;
}

mtf_status mtf_learned_train(mtf_system sys, int32_t steps, double lr, int32_t batch, int32_t K, uint64_t seed,
                             double* loss_first, double* loss_last, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    learned_train(sys, steps, lr, batch, K, seed, loss_first, loss_last, static_cast<cudaStream_t>(stream));
  });
}

mtf_status mtf_learned_fit(mtf_system sys, int32_t n_val, const double* dirs, const double* pols, int32_t rounds,
                           int32_t steps_per_round, double lr, int32_t batch, int32_t K, uint64_t seed,
                           mtf_learned_report* report, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(sys->learned, MTF_ERR_ARG, "the learned correction has not been initialised");
    MTF_REQUIRE(n_val >= 1 && dirs && pols && rounds >= 0 && steps_per_round >= 0, MTF_ERR_ARG,
                "n_val >= 1, rounds >= 0, steps_per_round >= 0 and non-null plane waves");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf<double> dd, dp, b, x;
    upload_waves(dd, dp, n_val, dirs, pols, s);
    b.alloc(size_t(sys->mesh->n_total) * n_val * 2);
    x.alloc(b.n);
    launch_rhs(sys, n_val, dd.p, dp.p, b.p, s);
    // iterations of a validation solve; a solve that misses the tolerance
    // counts as no improvement
    auto validate = [&]() {
      mtf_solve_stats st{};
      const mtf_status r = solve(sys, n_val, b.p, x.p, &st, s);
      MTF_CUDA(cudaStreamSynchronize(s));
      if (r == MTF_ERR_NOCONV || r == MTF_ERR_NAN || !st.converged) return INT32_MAX;
      MTF_REQUIRE(r == MTF_OK, r, "validation solve failed");
      return int(st.iterations);
    };
    mtf_learned_report rep{};
    sys->opt.learned = 0;
    rep.plain_iterations = validate();
    rep.best_iterations = rep.plain_iterations;
    std::vector<float> best(static_cast<size_t>(learned_param_count(sys)));
    sys->opt.learned = 1;
    for (int r = 1; r <= rounds; ++r) {
      double l0 = 0, l1 = 0;
      learned_train(sys, steps_per_round, lr, batch, K, seed, &l0, &l1, s);
      if (r == 1) rep.loss_first = l0;
      rep.loss_last = l1;
      rep.rounds = r;
      const int it = validate();
      if (it < rep.best_iterations) {
        rep.best_iterations = it;
        rep.best_round = r;
        learned_get_params(sys, best.data(), s);
      }
    }
    if (rep.best_round > 0) learned_set_params(sys, best.data(), s);
    rep.enabled = rep.best_round > 0 ? 1 : 0;
    sys->opt.learned = rep.enabled;
    if (report) *report = rep;
  });
}

mtf_status mtf_learned_enable(mtf_system sys, int32_t on) {
  return guarded([&] {
    require_learned_system(sys);
    sys->opt.learned = on ? 1 : 0;
  });
}

mtf_status mtf_learned_apply(mtf_system sys, const void* r, void* z, int32_t nrhs, void* stream) {
  return guarded([&] {
    require_learned_system(sys);
    MTF_REQUIRE(sys->learned, MTF_ERR_ARG, "the learned correction has not been initialised");
    MTF_REQUIRE(r && z && r != z && nrhs >= 1, MTF_ERR_ARG, "null or overlapping argument, or nrhs < 1");
    const int64_t n = sys->mesh->n_total;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    launch_osrc_apply_f32(sys, static_cast<const float*>(r), n, static_cast<float*>(z), n, nrhs, s);
    learned_apply_inplace(sys, static_cast<const float*>(r), n, static_cast<float*>(z), n, nrhs, s);
  });
}

mtf_status mtf_nearfield(mtf_system sys, const void* x, int32_t nrhs, const double* points, const int32_t* domains,
                         int32_t n_pts, void* f_out, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && x && points && domains && f_out, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1 && n_pts >= 1, MTF_ERR_ARG, "nrhs and n_pts must be >= 1");
    const int nd = sys->mesh->nd;
    for (int32_t p = 0; p < n_pts; ++p)
      MTF_REQUIRE(domains[p] >= 0 && domains[p] < nd && std::isfinite(points[3 * p]) &&
                      std::isfinite(points[3 * p + 1]) && std::isfinite(points[3 * p + 2]),
                  MTF_ERR_ARG, "point with a subdomain out of range or a non-finite coordinate");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf<double> dp;
    DevBuf<int32_t> dd;
    dp.alloc(size_t(3) * n_pts);
    dd.alloc(size_t(n_pts));
    MTF_CUDA(cudaMemcpyAsync(dp.p, points, size_t(3) * n_pts * sizeof(double), cudaMemcpyHostToDevice, s));
    MTF_CUDA(cudaMemcpyAsync(dd.p, domains, size_t(n_pts) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    launch_nearfield(sys, static_cast<const double*>(x), nrhs, dp.p, dd.p, n_pts, static_cast<double*>(f_out), s);
  });
}

mtf_status mtf_farfield(mtf_system sys, const void* x, int32_t nrhs, const double* obs_dirs, int32_t n_obs,
                        void* f_out, void* stream) {
  return guarded([&] {
    MTF_REQUIRE(sys && x && obs_dirs && f_out, MTF_ERR_ARG, "null argument");
    MTF_REQUIRE(nrhs >= 1 && n_obs >= 1, MTF_ERR_ARG, "need nrhs >= 1 and n_obs >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevBuf<double> d_obs;
    upload_small(d_obs, obs_dirs, size_t(n_obs) * 3, s);
    launch_farfield(sys, static_cast<const double*>(x), nrhs, d_obs.p, n_obs, static_cast<double*>(f_out), s);
    MTF_CUDA(cudaStreamSynchronize(s));
  });
}

void mtf_system_destroy(mtf_system sys) {
  if (!sys) return;
  destroy_gmres(sys->gw);
  destroy_gmres32(sys->gw32);
  destroy_block32(sys->bw);
  destroy_tc(sys->tc);
  destroy_tt(sys->tt);
  destroy_learned(sys->learned);
  delete sys;
}

const char* mtf_status_string(mtf_status s) {
  switch (s) {
    case MTF_OK: return "ok";
    case MTF_ERR_ARG: return "invalid argument";
    case MTF_ERR_MESH: return "invalid mesh";
    case MTF_ERR_CUDA: return "CUDA error";
    case MTF_ERR_OOM: return "out of device memory";
    case MTF_ERR_NOCONV: return "solver did not converge";
    case MTF_ERR_NAN: return "non-finite value";
    case MTF_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* mtf_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
