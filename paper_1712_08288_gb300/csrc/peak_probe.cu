// peak_probe.cu -- lbm_probe_fp64_rate: the device's FP64 fused multiply-add rate,
// measured with a plain FMA loop, the denominator the FP64 sweep (bound by the
// FP64 pipe on this GPU, not by HBM) is reported against.  No device setting is
// changed; the probe allocates 8 bytes and frees them.
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kChains = 8;        // independent FMA chains per thread (hides the FMA latency)
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_loop(double *sink, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[0] = s;   // never true: keeps the chains live
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_probe_fp64_rate(double *gflops) {
  using namespace lbm;
  if (!gflops) return LBM_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_loop, kProbeThreads, 0);
  if (sms <= 0 || per_sm <= 0) return LBM_ECUDA;
  const int blocks = sms * per_sm;
  const int iters = 1 << 14;
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    cudaEventRecord(e0);
    fp64_fma_loop<<<blocks, kProbeThreads>>>(sink, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return LBM_ECUDA;
  const double flops = 2.0 * kChains * (double)iters * blocks * kProbeThreads;
  *gflops = flops / (best * 1e-3) / 1e9;
  return LBM_OK;
}
