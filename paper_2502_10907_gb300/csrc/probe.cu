// Arithmetic-peak probes: the rates that bound the assembly kernels (FP32 and
// FP64 fused multiply-add, and the special-function unit that evaluates the
// sines and cosines of the Green's function phases), measured on the device
// rather than taken from unit counts.  Each probe runs independent dependency
// chains per thread (enough in flight to cover the pipe latency) over a grid
// of several CTAs per SM, and is timed with CUDA events on the caller's
// stream after one warm-up launch.  The chains' results are folded into one
// store per thread so that the compiler keeps the work.
#include <cuda_runtime.h>

#include "common.h"

namespace mtf {

constexpr int kProbeChains = 8;

template <class T>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T b, T c, T* __restrict__ sink) {
  T a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
  }
  T r = 0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) r += a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void __launch_bounds__(256) k_probe_sfu(int iters, float* __restrict__ sink) {
  float a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = float(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __sinf(a[k]);
  }
  float r = 0.f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) r += a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// rates[0]: FP32 FLOP/s (an FMA counts 2), rates[1]: FP64 FLOP/s,
// rates[2]: special-function results (__sinf) per second
void probe_peaks(double* rates, cudaStream_t s) {
  int dev = 0, sms = 0;
  MTF_CUDA(cudaGetDevice(&dev));
  MTF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = 8 * sms, block = 256;
  const double threads = double(grid) * block;
  DevBuf<double> sink;
  sink.alloc(size_t(grid) * block);
  cudaEvent_t e0, e1;
  MTF_CUDA(cudaEventCreate(&e0));
  MTF_CUDA(cudaEventCreate(&e1));
  auto timed = [&](auto launch) {
    launch();  // warm-up
    MTF_CUDA(cudaEventRecord(e0, s));
    launch();
    MTF_CUDA(cudaEventRecord(e1, s));
    MTF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MTF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return double(ms) * 1e-3;
  };
  const int it32 = 4096, it64 = 128, itsfu = 1024;
  const double t32 = timed([&] {
    MTF_LAUNCH(KID_MISC, s, k_probe_fma<float><<<grid, block, 0, s>>>(it32, 0.999f, 1e-4f,
                                                                      reinterpret_cast<float*>(sink.p)));
  });
  const double t64 = timed([&] {
    MTF_LAUNCH(KID_MISC, s, k_probe_fma<double><<<grid, block, 0, s>>>(it64, 0.999, 1e-4, sink.p));
  });
  const double tsf = timed([&] {
    MTF_LAUNCH(KID_MISC, s, k_probe_sfu<<<grid, block, 0, s>>>(itsfu, reinterpret_cast<float*>(sink.p)));
  });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  rates[0] = 2.0 * kProbeChains * double(it32) * threads / t32;
  rates[1] = 2.0 * kProbeChains * double(it64) * threads / t64;
  rates[2] = double(kProbeChains) * double(itsfu) * threads / tsf;
}

}  // namespace mtf
