// aux_kernels.cu -- kernels off the time-step path: equilibrium initialisation
// (Eq. 42), population import/export, FP64 moments (Appendix, rho and rho0 u) and
// the FP64 block reductions behind the error norms (Sec. 3.1, E_r).
//
// All of them read populations through the AA layout of the sweep: after an even
// number of steps f_i(x) sits in slot i of x, after an odd number in slot opp(i)
// of x - e_i, or in the link buffer for a cut link.  They compute in double
// whatever the storage type.
#include "common.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

template <class L, class T>
__global__ void init_eq_kernel(AuxArgs a, const double *rho, const double *u) {
  T *pop = static_cast<T *>(a.pop);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    if (a.cls[n] == kSolid) {
      for (int i = 0; i < L::Q; ++i) Storage<T>::store(pop + (long long)i * a.S + n, 0.0);
      continue;
    }
    const double drho = rho ? rho[n] - a.rho0 : 0.0;
    double ux = 0, uy = 0, uz = 0;
    if (u) {
      ux = u[n * L::D];
      uy = u[n * L::D + 1];
      if (L::D == 3) uz = u[n * L::D + 2];
    }
    const double u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double cu = L::ex(i) * ux + L::ey(i) * uy + L::ez(i) * uz;
      // Eq. 42 minus w_i rho0, c_s^2 = 1/3
      const double geq = L::w(i) * (drho + a.rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2));
      Storage<T>::store(pop + (long long)i * a.S + n, geq);
    }
  }
}

template <class L, class T>
__global__ void get_pop_kernel(AuxArgs a, bool odd, double *f) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const bool solid = a.cls[n] == kSolid;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      double v = quiet_nan();
      if (!solid) v = L::w(i) * a.rho0 + (double)Storage<T>::load(population_address<L, T>(i, n, odd, a));
      f[(long long)i * a.N + n] = v;
    }
  }
}

template <class L, class T>
__global__ void set_pop_kernel(AuxArgs a, const double *f) {
  T *pop = static_cast<T *>(a.pop);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const bool solid = a.cls[n] == kSolid;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double v = solid ? 0.0 : f[(long long)i * a.N + n] - L::w(i) * a.rho0;
      Storage<T>::store(pop + (long long)i * a.S + n, v);
    }
  }
}

// density deviation and momentum of node n
template <class L, class T>
__device__ __forceinline__ void node_moments(const AuxArgs &a, const T *pop, long long n, bool odd,
                                             double &drho, double (&j)[3]) {
  drho = 0;
  j[0] = j[1] = j[2] = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double g = (double)Storage<T>::load(population_address<L, T>(i, n, odd, a));
    drho += g;
    j[0] += L::ex(i) * g;
    j[1] += L::ey(i) * g;
    j[2] += L::ez(i) * g;
  }
}

template <class L, class T>
__global__ void moments_kernel(AuxArgs a, bool odd, double *rho, double *u) {
  const T *pop = static_cast<const T *>(a.pop);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    if (a.cls[n] == kSolid) {
      if (rho) rho[n] = quiet_nan();
      if (u)
        for (int k = 0; k < L::D; ++k) u[n * L::D + k] = quiet_nan();
      continue;
    }
    double drho, j[3];
    node_moments<L, T>(a, pop, n, odd, drho, j);
    if (rho) rho[n] = a.rho0 + drho;
    if (u)
      for (int k = 0; k < L::D; ++k) u[n * L::D + k] = j[k] / a.rho0 + 0.5 * a.g[k];
  }
}

constexpr int kNormThreads = 256;

template <class L, class T>
__global__ void __launch_bounds__(kNormThreads)
    norm_partials_kernel(AuxArgs a, bool odd, const double *u_ref, double *u_prev,
                         double *partials) {
  const T *pop = static_cast<const T *>(a.pop);
  double acc[kNormFields];
#pragma unroll
  for (int k = 0; k < kNormFields; ++k) acc[k] = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    if (a.cls[n] == kSolid) continue;
    double drho, j[3];
    node_moments<L, T>(a, pop, n, odd, drho, j);
    const double rho = a.rho0 + drho;
    if (!isfinite(rho)) acc[9] += 1.0;
    acc[3] += rho;
    acc[4] += j[0];
    acc[5] += j[1];
    acc[6] += j[2];
#pragma unroll
    for (int k = 0; k < L::D; ++k) {
      const double uk = j[k] / a.rho0 + 0.5 * a.g[k];
      if (u_ref) {
        const double r = u_ref[n * L::D + k];
        const double df = r - uk;
        acc[0] += df * df;
        acc[1] += r * r;
        acc[2] = fmax(acc[2], fabs(df));
      }
      const double dp = uk - u_prev[n * L::D + k];
      acc[7] += dp * dp;
      acc[8] += uk * uk;
      u_prev[n * L::D + k] = uk;
    }
  }
  // block reduction (fixed order -> deterministic)
  __shared__ double sh[kNormThreads / 32][kNormFields];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNormFields; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = (k == 2) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNormFields) {
    const int k = threadIdx.x;
    double v = sh[0][k];
    for (int w = 1; w < kNormThreads / 32; ++w) v = (k == 2) ? fmax(v, sh[w][k]) : v + sh[w][k];
    partials[(long long)blockIdx.x * kNormFields + k] = v;
  }
}

__global__ void norm_finish_kernel(const double *partials, int n_blocks, double *out) {
  // one block; thread k < kNormFields reduces field k over the blocks in order
  const int k = threadIdx.x;
  if (k >= kNormFields) return;
  double v = (k == 2) ? 0.0 : 0.0;
  for (int b = 0; b < n_blocks; ++b) {
    const double w = partials[(long long)b * kNormFields + k];
    v = (k == 2) ? fmax(v, w) : v + w;
  }
  out[k] = v;
}

int aux_blocks(long long N) {
  long long b = (N + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int norm_blocks_for(long long N) {
  long long b = (N + kNormThreads - 1) / kNormThreads;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_init_equilibrium(int lattice, int precision, const AuxArgs &a,
                                    const double *rho, const double *u, cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      init_eq_kernel<L, T><<<aux_blocks(a.N), 256, 0, st>>>(a, rho, u);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_get_populations(int lattice, int precision, const AuxArgs &a, bool odd,
                                   double *f, cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      get_pop_kernel<L, T><<<aux_blocks(a.N), 256, 0, st>>>(a, odd, f);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_set_populations(int lattice, int precision, const AuxArgs &a,
                                   const double *f, cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      set_pop_kernel<L, T><<<aux_blocks(a.N), 256, 0, st>>>(a, f);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_moments(int lattice, int precision, const AuxArgs &a, bool odd, double *rho,
                           double *u, cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      moments_kernel<L, T><<<aux_blocks(a.N), 256, 0, st>>>(a, odd, rho, u);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_norm_partials(int lattice, int precision, const AuxArgs &a, bool odd,
                                 const double *u_ref, double *u_prev, double *partials,
                                 int n_blocks, cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      norm_partials_kernel<L, T><<<n_blocks, kNormThreads, 0, st>>>(a, odd, u_ref, u_prev,
                                                                      partials);
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_norm_finish(const double *partials, int n_blocks, double *out,
                               cudaStream_t st) {
  norm_finish_kernel<<<1, 32, 0, st>>>(partials, n_blocks, out);
  return cudaGetLastError();
}

}  // namespace lbm
