// Per-kernel accounting: launch counts always, and (when enabled) device
// durations from CUDA events recorded on the launching stream around each
// launch.  Used by the benchmark for the roofline of the dominant kernel and
// for the number of library kernels launched in a timed region.
#include <vector>

#include <atomic>
#include <mutex>

#include "common.h"

namespace mtf {

static const char* kNames[KID_COUNT] = {
    "regular64", "singular64", "exchange_values", "rhs", "matvec64", "gmres_dots",
    "gmres_axpy", "gmres_norm_scale", "gmres_sub", "farfield", "split_block",
    "regular32", "matvec32", "osrc_apply", "mlp", "misc", "matvec32_combine", "osrc_combine",
    "matvec_tc", "matvec_tc_prep", "matvec_tc_combine", "tc_tile", "block_cholesky", "block_xform",
    "basis_store", "osrc_form_prep", "osrc_form_mma", "gs_prep", "block_gram"};

// Counters shared by every host thread that launches library kernels (the
// batched solve drives its instances from several threads): launch counts are
// atomic, the rest is guarded by mu.
struct Prof {
  std::mutex mu;
  std::atomic<bool> on{false};
  std::atomic<int64_t> launches[KID_COUNT] = {};
  double ms[KID_COUNT] = {};
  double bytes[KID_COUNT] = {};  // algorithmic bytes declared by the launch sites
  struct Rec {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    cudaEvent_t e;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      MTF_CUDA(cudaEventCreate(&e));
    }
    return e;
  }
};
static Prof g_prof;
static thread_local cudaEvent_t t_begin = nullptr;

void prof_begin(int kid, cudaStream_t s) {
  (void)kid;
  if (!g_prof.on.load(std::memory_order_relaxed)) return;
  {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    t_begin = g_prof.get();
  }
  MTF_CUDA(cudaEventRecord(t_begin, s));
}

void prof_end(int kid, cudaStream_t s) {
  g_prof.launches[kid].fetch_add(1, std::memory_order_relaxed);
  if (!g_prof.on.load(std::memory_order_relaxed) || !t_begin) return;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  cudaEvent_t e = g_prof.get();
  MTF_CUDA(cudaEventRecord(e, s));
  g_prof.pending.push_back({kid, t_begin, e});
  t_begin = nullptr;
}

static void resolve() {
  for (auto& r : g_prof.pending) {
    MTF_CUDA(cudaEventSynchronize(r.b));
    float ms = 0;
    MTF_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    g_prof.ms[r.kid] += ms;
    g_prof.pool.push_back(r.a);
    g_prof.pool.push_back(r.b);
  }
  g_prof.pending.clear();
}

void prof_enable(bool on) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!on) resolve();
  g_prof.on = on;
}

void prof_bytes(int kid, double b) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.bytes[kid] += b;
}

void prof_read(int n, int64_t* launches, double* ms, double* bytes) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  resolve();
  for (int k = 0; k < n && k < KID_COUNT; ++k) {
    if (launches) launches[k] = g_prof.launches[k].load();
    if (ms) ms[k] = g_prof.ms[k];
    if (bytes) bytes[k] = g_prof.bytes[k];
    g_prof.launches[k] = 0;
    g_prof.ms[k] = 0;
    g_prof.bytes[k] = 0;
  }
}

const char* kernel_name(int kid) { return kid >= 0 && kid < KID_COUNT ? kNames[kid] : "?"; }

}  // namespace mtf
