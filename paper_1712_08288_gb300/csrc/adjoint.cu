// adjoint.cu -- discrete adjoint (reverse mode) of the fused time step, for a
// velocity-mismatch loss J = sum over masked fluid nodes of |u(x, T) - u*(x)|^2.
//
// Kernels:
//   export_state   AA layout (any storage) -> natural layout deviations g[i*N+n]
//                  in the compute type (checkpoints, segment states);
//   import_state   natural layout -> AA even layout (restore a checkpoint);
//   loss           J and lambda(T) = dJ/df(T) = 2 (u - u*).e_i / rho0;
//   adjoint_step   lambda(t) from lambda(t+1) and the pre-collision state f(t),
//                  accumulating dJ/ds_k, dJ/dq and dJ/dphi of every link.
//
// The adjoint of one step, per fluid node x (Sec. 2 and Appendix restated in
// reverse):
//   advection (Eq. 2.2b): the adjoint of f'_i(x) gathers lambda_i(x + e_i) from
//     fluid neighbours;
//   boundary (Eq. 2.13): for a cut link (x, d), i = opp(d), the new f_i(x) is
//     (1-b) f_i + bA f_d + bB f'_i + bC f'_d + bW, so lambda_i(x) of the next step
//     is sent back with those weights, and d/dgamma, d/dphi of the same
//     expression give the link gradients;
//   collision (Appendix, MRT): with mu = M^-T lambda' (M^-T = diag(1/|M_k|^2) M),
//     nu_k = (1 - s_k) mu_k for non-conserved rows and
//     nu_k = mu_k + sum_l s_l (d meq_l / d m_k) mu_l for rho and j, where the
//     derivatives of the equilibrium moments are obtained by evaluating the same
//     meq() in forward-mode dual numbers; lambda(t) = M^T nu + boundary terms, and
//     dJ/ds_k += mu_k * (-(m_k - meq_k)).
#include "sweep.cuh"

namespace lbm {

// ---- forward-mode dual numbers with four partials (rho, j_x, j_y, j_z) ----------
template <class C>
struct Dual4 {
  C v, d[4];
  __device__ __forceinline__ Dual4() {}
  __device__ __forceinline__ Dual4(double x) : v(C(x)) { d[0] = d[1] = d[2] = d[3] = C(0); }
  __device__ __forceinline__ static Dual4 var(C x, int k) {
    Dual4 r(0.0);
    r.v = x;
    r.d[k] = C(1);
    return r;
  }
};
template <class C>
__device__ __forceinline__ Dual4<C> operator+(const Dual4<C> &a, const Dual4<C> &b) {
  Dual4<C> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <class C>
__device__ __forceinline__ Dual4<C> operator-(const Dual4<C> &a, const Dual4<C> &b) {
  Dual4<C> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <class C>
__device__ __forceinline__ Dual4<C> operator-(const Dual4<C> &a) {
  Dual4<C> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = -a.d[k];
  return r;
}
template <class C>
__device__ __forceinline__ Dual4<C> operator*(const Dual4<C> &a, const Dual4<C> &b) {
  Dual4<C> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}

namespace {

constexpr int kAdjThreads = 128;

__device__ __forceinline__ void atomic_add_double(double *p, double v) { atomicAdd(p, v); }

template <class L, class T, class C>
__global__ void export_state_kernel(AuxArgs a, bool odd, C *out) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const bool solid = a.cls[n] == kSolid;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      out[(long long)i * a.N + n] =
          solid ? C(0) : C(Storage<T>::load(population_address<L, T>(i, n, odd, a)));
  }
}

template <class L, class T, class C>
__global__ void import_state_kernel(AuxArgs a, const C *in) {
  T *pop = static_cast<T *>(a.pop);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const bool solid = a.cls[n] == kSolid;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      Storage<T>::store(pop + (long long)i * a.S + n, solid ? C(0) : in[(long long)i * a.N + n]);
  }
}

// J and lambda(T); u = j/rho0 + g/2 from the natural-layout deviations
template <class L, class C>
__global__ void loss_kernel(AuxArgs a, const C *g, const uint8_t *mask, const double *u_target,
                            C *lam, double *J) {
  double acc = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < a.N;
       n += (long long)gridDim.x * blockDim.x) {
    const bool on = a.cls[n] != kSolid && mask[n];
    double j[3] = {0.0, 0.0, 0.0};
    if (on) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const double v = (double)g[(long long)i * a.N + n];
        j[0] += L::ex(i) * v;
        j[1] += L::ey(i) * v;
        j[2] += L::ez(i) * v;
      }
    }
    double diff[3] = {0.0, 0.0, 0.0};
    if (on)
      for (int k = 0; k < L::D; ++k) {
        diff[k] = j[k] / a.rho0 + 0.5 * a.g[k] - u_target[n * L::D + k];
        acc += diff[k] * diff[k];
      }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double v = 2.0 / a.rho0 * (L::ex(i) * diff[0] + L::ey(i) * diff[1] + L::ez(i) * diff[2]);
      lam[(long long)i * a.N + n] = C(v);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomic_add_double(J, acc);
}

struct AdjGeo {
  const double *link_q;       // wall fraction per link (device order)
  const double *link_ephi;    // e_i . phi per link, i = opp(d)
  double *grad_q;             // accumulated dJ/dq per link
  double *grad_phi;           // accumulated dJ/dphi per link (3 each)
  double *grad_s;             // accumulated dJ/ds_k (Q)
  double c0, c1, c2, b, rho0;
  double s[19];               // relaxation rates
};

template <class L, class C>
__global__ void __launch_bounds__(kAdjThreads)
    adjoint_step_kernel(const SweepArgs<C> sa, AuxArgs a, AdjGeo ag, const C *__restrict__ f,
                        const C *__restrict__ lam_in, C *__restrict__ lam_out) {
  constexpr int Q = L::Q;
  const long long N = a.N;
  C gs[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) gs[k] = C(0);
  const LinkCoef<C> *coef = static_cast<const LinkCoef<C> *>(sa.geo.coef);
  const C ir0 = sa.inv_rho0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const uint8_t cls = a.cls[n];
    if (cls == kSolid) {
#pragma unroll
      for (int i = 0; i < Q; ++i) lam_out[(long long)i * N + n] = C(0);
      continue;
    }
    const int x = (int)(n % a.nx);
    const long long r = n / a.nx;
    const int y = (int)(r % a.ny), z = (int)(r / a.ny);
    C g[Q], gp[Q], lp[Q], lpre[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      g[i] = f[(long long)i * N + n];
      lpre[i] = C(0);
    }
    C drho;
    collide<L, C>(g, gp, sa, drho);
    // advection transpose: gather lambda_i(x + e_i) from fluid neighbours
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const long long nb = wrap_index(x, y, z, L::ex(i), L::ey(i), L::ez(i), a.nx, a.ny, a.nz, a.sy, a.sz);
      lp[i] = a.cls[nb] != kSolid ? lam_in[(long long)i * N + nb] : C(0);
    }
    // boundary transpose and link gradients (Eq. 2.13)
    if (cls == kBoundary) {
      const int bi = a.bidx[n];
      const uint32_t mask = a.bmask[bi];
      const int off = a.boff[bi];
#pragma unroll
      for (int dd = 1; dd < Q; ++dd) {
        if (mask & (1u << dd)) {
          const int k = off + __popc(mask & ((1u << dd) - 1u));
          const LinkCoef<C> c = coef[k];
          const int i = L::opp(dd);
          const C av = lam_in[(long long)i * N + n];
          lp[i] += c.bb * av;
          lp[dd] += c.c * av;
          lpre[i] += sa.one_minus_b * av;
          lpre[dd] += c.a * av;
          const double q = ag.link_q[k];
          const double l = ag.c0 + ag.c1 * q + ag.c2 * q * q;
          const double lq = ag.c1 + 2.0 * ag.c2 * q;
          const double inv = 1.0 / (1.0 + l), inv2 = inv * inv;
          const double dA = (-2.0 * (1.0 + l) + 2.0 * q * lq) * inv2;
          const double dB = lq * inv2;
          const double dC = (2.0 * (1.0 + l) - lq - 2.0 * q * lq) * inv2;
          const double E = L::w(i) * ag.rho0 * 3.0 * ag.link_ephi[k];   // w rho0 e.phi / c_s^2
          const double dW = -2.0 * lq * inv2 * E;
          const double da = (double)av * ag.b;
          ag.grad_q[k] += da * (dA * (double)g[dd] + dB * (double)gp[i] + dC * (double)gp[dd] + dW);
          const double wphi = da * 2.0 * inv * L::w(i) * ag.rho0 * 3.0;
          ag.grad_phi[3 * k + 0] += wphi * L::ex(i);
          ag.grad_phi[3 * k + 1] += wphi * L::ey(i);
          ag.grad_phi[3 * k + 2] += wphi * L::ez(i);
        }
      }
    }
    // collision transpose
    C drho_m = g[0];
    C jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) drho_m += g[i];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      jx = madd(jx, L::ex(i), g[i]);
      jy = madd(jy, L::ey(i), g[i]);
      jz = madd(jz, L::ez(i), g[i]);
    }
    const Dual4<C> dr = Dual4<C>::var(drho_m, 0), dx = Dual4<C>::var(jx, 1), dy = Dual4<C>::var(jy, 2),
                   dz = Dual4<C>::var(jz, 3);
    const Dual4<C> ir = Dual4<C>((double)ir0);
    C mu[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      C m = C(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) m = madd(m, L::M(k, i), lp[i]);
      mu[k] = m * C(1.0 / row_norm2<L>(k));
    }
    C nu_c[4] = {mu[0], C(0), C(0), C(0)};    // rho, j_x, j_y, j_z rows
    constexpr int jr[3] = {3, 5, 7};
    nu_c[1] = mu[jr[0]];
    nu_c[2] = mu[jr[1]];
    if (L::D == 3) nu_c[3] = mu[jr[2]];
    C nu[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      if (Rows<L>::cons(k)) { nu[k] = C(0); continue; }
      const C sk = C(ag.s[k]);
      const Dual4<C> me = meq(L{}, k, dr, dx, dy, dz, ir);
      C mk = C(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) mk = madd(mk, L::M(k, i), g[i]);
      gs[k] += mu[k] * (me.v - mk);                  // d m'_k / d s_k = -(m_k - meq_k)
      nu[k] = (C(1) - sk) * mu[k];
      const C smu = sk * mu[k];
#pragma unroll
      for (int c = 0; c < 4; ++c) nu_c[c] += smu * me.d[c];
    }
    nu[0] = nu_c[0];
    nu[jr[0]] = nu_c[1];
    nu[jr[1]] = nu_c[2];
    if (L::D == 3) nu[jr[2]] = nu_c[3];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      C v = lpre[i];
#pragma unroll
      for (int k = 0; k < Q; ++k) v = madd(v, L::M(k, i), nu[k]);
      lam_out[(long long)i * N + n] = v;
    }
  }
  // dJ/ds: block reduction, then one FP64 atomic per row and block
  __shared__ double sh[kAdjThreads / 32][Q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    double v = (double)gs[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < Q) {
    double v = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) v += sh[w][threadIdx.x];
    atomic_add_double(ag.grad_s + threadIdx.x, v);
  }
}

int adj_blocks(long long N) {
  long long b = (N + kAdjThreads - 1) / kAdjThreads;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_export_state(int lattice, int precision, const AuxArgs &a, bool odd, void *out,
                                cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      using C = typename Storage<T>::C;
      export_state_kernel<L, T, C><<<adj_blocks(a.N), 256, 0, st>>>(a, odd, static_cast<C *>(out));
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_import_state(int lattice, int precision, const AuxArgs &a, const void *in,
                                cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      using C = typename Storage<T>::C;
      import_state_kernel<L, T, C><<<adj_blocks(a.N), 256, 0, st>>>(a, static_cast<const C *>(in));
      return cudaGetLastError();
    });
  });
}

cudaError_t launch_loss(int lattice, int precision, const AuxArgs &a, const void *g,
                        const uint8_t *mask, const double *u_target, void *lam, double *J,
                        cudaStream_t st) {
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    if (precision == 0)
      loss_kernel<L, double><<<adj_blocks(a.N), 256, 0, st>>>(a, static_cast<const double *>(g), mask,
                                                              u_target, static_cast<double *>(lam), J);
    else
      loss_kernel<L, float><<<adj_blocks(a.N), 256, 0, st>>>(a, static_cast<const float *>(g), mask,
                                                             u_target, static_cast<float *>(lam), J);
    return cudaGetLastError();
  });
}

cudaError_t launch_adjoint_step(int lattice, int precision, const SweepArgs<double> &a64,
                                const SweepArgs<float> &a32, const AuxArgs &a, const double *link_q,
                                const double *link_ephi, double *grad_q, double *grad_phi,
                                double *grad_s, double c0, double c1, double c2, double b,
                                double rho0, const double *s, const void *f, const void *lam_in,
                                void *lam_out, cudaStream_t st) {
  AdjGeo ag{link_q, link_ephi, grad_q, grad_phi, grad_s, c0, c1, c2, b, rho0, {0}};
  for (int k = 0; k < 19; ++k) ag.s[k] = s[k];
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    if (precision == 0)
      adjoint_step_kernel<L, double><<<adj_blocks(a.N), kAdjThreads, 0, st>>>(
          a64, a, ag, static_cast<const double *>(f), static_cast<const double *>(lam_in),
          static_cast<double *>(lam_out));
    else
      adjoint_step_kernel<L, float><<<adj_blocks(a.N), kAdjThreads, 0, st>>>(
          a32, a, ag, static_cast<const float *>(f), static_cast<const float *>(lam_in),
          static_cast<float *>(lam_out));
    return cudaGetLastError();
  });
}

}  // namespace lbm
