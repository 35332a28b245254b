// C-ABI of libmtf (declared in include/mtf.h).  Every entry point converts
// internal errors into an mtf_status and records a message for
// mtf_last_error(); nothing throws across the boundary.
#include <cmath>
#include <complex>
#include <cstring>
#include <string>

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
  buf.alloc(n);
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
    DevBuf<double> dd, dp, b;
    upload_waves(dd, dp, nrhs, dirs, pols, s);
    b.alloc(size_t(sys->mesh->n_total) * nrhs * 2);
    launch_rhs(sys, nrhs, dd.p, dp.p, b.p, s);
    st = solve(sys, nrhs, b.p, static_cast<double*>(x_out), stats, s);
    MTF_CUDA(cudaStreamSynchronize(s));
    if (st == MTF_ERR_NOCONV) set_last_error("GMRES did not reach the tolerance within max_iter");
    if (st == MTF_ERR_NAN) set_last_error("non-finite residual in GMRES");
  });
  return g != MTF_OK ? g : st;
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
