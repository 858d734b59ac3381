// common.cuh -- storage conversions and periodic neighbour indexing used by the
// kernels of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "lattice.h"
#include "lbm_internal.h"

namespace lbm {

// storage type -> compute type and conversions
template <class T>
struct Storage;
template <>
struct Storage<double> {
  using C = double;
  static __device__ __forceinline__ double load(const double *p) { return *p; }
  static __device__ __forceinline__ void store(double *p, double v) { *p = v; }
};
template <>
struct Storage<float> {
  using C = float;
  static __device__ __forceinline__ float load(const float *p) { return *p; }
  static __device__ __forceinline__ void store(float *p, float v) { *p = v; }
};
template <>
struct Storage<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ float load(const __nv_bfloat16 *p) {
    return __bfloat162float(*p);
  }
  static __device__ __forceinline__ void store(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
  }
};
template <>
struct Storage<__half> {
  using C = float;
  static __device__ __forceinline__ float load(const __half *p) { return __half2float(*p); }
  static __device__ __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
};

// Linear index of the periodic image of (x+dx, y+dy, z+dz), |d| <= 1.  The field
// is invariant under the translation (nx, sy, sz) with 0 <= sy < ny, 0 <= sz < nz
// and under (0, ny, 0), (0, 0, nz); one correction per axis is then enough.
__device__ __forceinline__ long long wrap_index(int x, int y, int z, int dx, int dy, int dz,
                                                int nx, int ny, int nz, int sy, int sz) {
  int xs = x + dx, ys = y + dy, zs = z + dz;
  if (xs < 0) {
    xs += nx;
    ys += sy;
    zs += sz;
  } else if (xs >= nx) {
    xs -= nx;
    ys -= sy;
    zs -= sz;
  }
  if (ys < 0) ys += ny;
  else if (ys >= ny) ys -= ny;
  if (zs < 0) zs += nz;
  else if (zs >= nz) zs -= nz;
  return xs + (long long)nx * (ys + (long long)ny * zs);
}

// Address of f_i(x_n, t) in the AA layout: after an even number of steps slot i of
// x_n; after an odd number slot opp(i) of x_n - e_i, except for a cut link
// (x_n - e_i solid), whose value sits in the link buffer.
template <class L, class T>
__device__ __forceinline__ const T *population_address(int i, long long n, bool odd,
                                                       const AuxArgs &a) {
  const T *pop = static_cast<const T *>(a.pop);
  if (!odd) return pop + (long long)i * a.S + n;
  const int d = L::opp(i);
  if (d != i && a.cls[n] == kBoundary) {
    const int b = a.bidx[n];
    const uint32_t m = a.bmask[b];
    if ((m >> d) & 1u)
      return static_cast<const T *>(a.lnk) + a.boff[b] + __popc(m & ((1u << d) - 1u));
  }
  const int x = (int)(n % a.nx);
  const long long r = n / a.nx;
  const int y = (int)(r % a.ny), z = (int)(r / a.ny);
  return pop + (long long)d * a.S +
         wrap_index(x, y, z, -L::ex(i), -L::ey(i), -L::ez(i), a.nx, a.ny, a.nz, a.sy, a.sz);
}

// dispatch helper: storage type for an lbm_precision value
template <class F>
__host__ inline cudaError_t with_storage(int precision, F &&f) {
  switch (precision) {
    case 0: return f((double *)nullptr);
    case 1: return f((float *)nullptr);
    case 2: return f((__nv_bfloat16 *)nullptr);
    case 3: return f((__half *)nullptr);
    default: return cudaErrorInvalidValue;
  }
}
template <class F>
__host__ inline cudaError_t with_lattice(int lattice, F &&f) {
  switch (lattice) {
    case 0: return f(D2Q9{});
    case 1: return f(D3Q19{});
    case 2: return f(D3Q15{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
