// noalloc.cu -- lbm_error_norms_noalloc: the error-norm reduction of
// lbm_error_norms with its block partial sums kept in a fixed, file-scope device
// array instead of memory obtained from cudaMalloc.
//
// Why: some callers cannot allocate device memory at the point where they want the
// norms -- applications that hand the whole device to their own memory pool at
// start-up, services that must run in a fixed, pre-declared memory footprint, and
// tight monitoring loops where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable.  lbm_error_norms allocates its scratch and
// staging buffers on first use and reads the result back to the host; this entry
// point allocates nothing, reads u_ref from the device and writes its result to a
// caller-owned device buffer on the context's stream.
//
// The scratch array (kNoAllocBlocks partial records, 80 KB) lives in every GPU that
// loads the library until the process exits.  All calls share it and it keeps the
// last call's contents; each call overwrites every record it reads, so nothing has
// to be cleared.  Calls whose kernels overlap on the GPU (other streams, other
// threads, other contexts) race on the array: issue them in order on one stream.
#include <mutex>

#include "../../include/lbm.h"
#include "common.cuh"

namespace lbm {
namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocBlocks = 1024;                     // partial records in the array
constexpr long long kNoAllocNodesPerBlock = 32768;       // nodes reduced by one block
constexpr long long kNoAllocMaxNodes = kNoAllocBlocks * kNoAllocNodesPerBlock;  // 33,554,432
constexpr int kFields = 8;  // sum|u_ref-u|^2, sum|u_ref|^2, max|u_ref-u|, sum rho, sum j (3), non-finite

static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks * kFields];

template <class L, class T>
__global__ void __launch_bounds__(kNoAllocThreads)
    noalloc_partials_kernel(AuxArgs a, bool odd, const double *u_ref, double *partials) {
  double acc[kFields];
#pragma unroll
  for (int k = 0; k < kFields; ++k) acc[k] = 0.0;
  const long long begin = (long long)blockIdx.x * kNoAllocNodesPerBlock;
  long long end = begin + kNoAllocNodesPerBlock;
  if (end > a.N) end = a.N;
  for (long long n = begin + threadIdx.x; n < end; n += kNoAllocThreads) {
    if (a.cls[n] == kSolid) continue;
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double g = (double)Storage<T>::load(population_address<L, T>(i, n, odd, a));
      drho += g;
      j[0] += L::ex(i) * g;
      j[1] += L::ey(i) * g;
      j[2] += L::ez(i) * g;
    }
    const double rho = a.rho0 + drho;
    if (!isfinite(rho)) acc[7] += 1.0;
    acc[3] += rho;
    acc[4] += j[0];
    acc[5] += j[1];
    acc[6] += j[2];
    if (u_ref) {
#pragma unroll
      for (int k = 0; k < L::D; ++k) {
        const double uk = j[k] / a.rho0 + 0.5 * a.g[k];
        const double df = u_ref[n * L::D + k] - uk;
        acc[0] += df * df;
        acc[1] += u_ref[n * L::D + k] * u_ref[n * L::D + k];
        acc[2] = fmax(acc[2], fabs(df));
      }
    }
  }
  __shared__ double sh[kNoAllocThreads / 32][kFields];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kFields; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = (k == 2) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kFields) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int w = 1; w < kNoAllocThreads / 32; ++w) v = (k == 2) ? fmax(v, sh[w][k]) : v + sh[w][k];
    partials[blockIdx.x * kFields + k] = v;
  }
}

// out: l2_rel, linf, mass, mom_x, mom_y, mom_z, non-finite count
__global__ void noalloc_finish_kernel(const double *partials, int n_blocks, bool have_ref,
                                      double *out) {
  __shared__ double tot[kFields];
  const int k = threadIdx.x;
  if (k < kFields) {
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) {
      const double w = partials[b * kFields + k];
      v = (k == 2) ? fmax(v, w) : v + w;
    }
    tot[k] = v;
  }
  __syncthreads();
  if (k == 0) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    out[0] = have_ref ? sqrt(tot[0]) / sqrt(tot[1]) : nan;
    out[1] = have_ref ? tot[2] : nan;
    out[2] = tot[3];
    out[3] = tot[4];
    out[4] = tot[5];
    out[5] = tot[6];
    out[6] = tot[7];
  }
}

// Device address of the scratch array, looked up once per device ordinal with
// that device current and kept for the life of the process.  The cache assumes
// the device's primary context lives as long as the process: after
// cudaDeviceReset (which unloads the library's device code and frees the array)
// the cached address is stale, so a caller that resets a device must not use this
// entry point on it again in the same process.
std::mutex g_mu;
double *g_scratch_addr[128] = {nullptr};

cudaError_t scratch_address(int device, double **out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (device < 0 || device >= 128) return cudaErrorInvalidDevice;
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

int error_norms_noalloc(int device, int lattice, int precision, const AuxArgs &a, bool odd,
                        const double *u_ref, double *out, cudaStream_t st, const char **why) {
  if (a.N > kNoAllocMaxNodes) {
    *why = "grid larger than the static scratch supports (33,554,432 nodes)";
    return LBM_EINVAL;
  }
  if (!out) {
    *why = "out_dev is NULL";
    return LBM_EINVAL;
  }
  DeviceGuard dg(device);
  double *scratch = nullptr;
  cudaError_t e = scratch_address(device, &scratch);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return LBM_ECUDA;
  }
  const int n_blocks = (int)((a.N + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock);
  e = with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      noalloc_partials_kernel<L, T><<<n_blocks, kNoAllocThreads, 0, st>>>(a, odd, u_ref, scratch);
      return cudaGetLastError();
    });
  });
  if (e == cudaSuccess) {
    noalloc_finish_kernel<<<1, 32, 0, st>>>(scratch, n_blocks, u_ref != nullptr, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return LBM_ECUDA;
  }
  return LBM_OK;
}

}  // namespace lbm
