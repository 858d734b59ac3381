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
//     nu_k = mu_k + sum_l s_l (d meq_l / d m_k) mu_l for rho and j, with the
//     derivatives of the closed-form equilibrium moments written out per lattice
//     (meq_adjoint); lambda(t) = M^T nu + boundary terms, and
//     dJ/ds_k += mu_k * (-(m_k - meq_k)).
// Adjoint entries of solid nodes are zero and stay zero (never written).
#include "sweep.cuh"

namespace lbm {

namespace {

constexpr int kAdjThreads = 128;
// resident blocks per SM the FP32 adjoint step is compiled for (register budget)
#ifndef LBM_ADJ_MINB_F32
#define LBM_ADJ_MINB_F32 6
#endif

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

// Link data of the adjoint step.  The gradients with respect to a link's wall
// fraction q and wall velocity phi are linear in two sums over the steps
// (Eq. 2.13 differentiated through l(q); a(t) the step's wall-velocity factor):
//   dJ/dq   = b sum_t lambda_i (A' f_d + B' f'_i + C' f'_d) + b W' sum_t a(t) lambda_i,
//   dJ/dphi = b 2 w_i rho0 e_i / ((1 + l) c_s^2) sum_t a(t) lambda_i,
// with ' = d/dq.  The kernel accumulates only sum_t a(t) lambda_i and the first sum,
// per link and in the compute type; the host folds in the other factors in FP64.
struct AdjGeo {
  const void *dcoef;          // LinkCoef<C> per link: (A', B', C', 0)
  void *acc;                  // 2 C per link: sum lambda_i, sum lambda_i (A' g_d + B' g'_i + C' g'_d)
};

// position of row k among the non-conserved rows
template <class L>
__host__ __device__ constexpr int nc_slot(int k) {
  int s = 0;
  for (int r = 0; r < k; ++r)
    if (!L::conserved(r)) ++s;
  return s;
}
static_assert(nc_slot<D3Q19>(19) <= 16 && nc_slot<D3Q15>(15) <= 16 && nc_slot<D2Q9>(9) <= 16,
              "at most 16 relaxed rows");

// Transposing warp reduction of 16 values per lane: at each of the offsets 16, 8,
// 4, 2 a lane keeps the half of its values that its lane bit selects and adds the
// partner's copy of that half; the pair (l, l^1) is combined last.  Lane l returns
// the warp sum of v[l >> 1]: 16 shuffles instead of 16 x 5.
template <class C>
__device__ __forceinline__ C warp_sum16(const C (&v)[16]) {
  const unsigned lane = threadIdx.x & 31u;
  const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u, b1 = lane & 2u;
  C a8[8], a4[4], a2[2];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    a8[j] = (b4 ? v[j + 8] : v[j]) + __shfl_xor_sync(0xffffffffu, b4 ? v[j] : v[j + 8], 16);
#pragma unroll
  for (int j = 0; j < 4; ++j)
    a4[j] = (b3 ? a8[j + 4] : a8[j]) + __shfl_xor_sync(0xffffffffu, b3 ? a8[j] : a8[j + 4], 8);
#pragma unroll
  for (int j = 0; j < 2; ++j)
    a2[j] = (b2 ? a4[j + 2] : a4[j]) + __shfl_xor_sync(0xffffffffu, b2 ? a4[j] : a4[j + 2], 4);
  C r = (b1 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? a2[0] : a2[1], 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

// sum_k smu_k * d meq_k / d(rho, j_x, j_y, j_z) for the equilibrium moments of
// meq() (deviation form), smu_k = s_k mu_k on the non-conserved rows
template <class C>
__device__ __forceinline__ void meq_adjoint(D2Q9, const C (&smu)[9], C jx, C jy, C, C ir0,
                                            C (&out)[4]) {
  out[0] = C(-2) * smu[1] + smu[2];
  const C a = C(6) * (smu[1] - smu[2]) * ir0;
  out[1] = a * jx - smu[4] + (C(2) * smu[7] * jx + smu[8] * jy) * ir0;
  out[2] = a * jy - smu[6] + (C(-2) * smu[7] * jy + smu[8] * jx) * ir0;
  out[3] = C(0);
}
template <class C>
__device__ __forceinline__ void meq_adjoint(D3Q19, const C (&smu)[19], C jx, C jy, C jz, C ir0,
                                            C (&out)[4]) {
  out[0] = C(-11) * smu[1] + C(3) * smu[2];
  const C a = (C(38) * smu[1] - C(11) * smu[2]) * ir0;    // e, eps: 19 j^2, -5.5 j^2
  const C px = (C(4) * smu[9] - C(2) * smu[10]) * ir0;    // 3p_xx, 3pi_xx along j_x
  const C pyz = (C(-2) * smu[9] + smu[10]) * ir0;         // 3p_xx, 3pi_xx along j_y, j_z
  const C w = (C(2) * smu[11] - smu[12]) * ir0;           // p_ww, pi_ww along j_y (-w along j_z)
  const C c23 = C(2.0 / 3.0);
  out[1] = (a + px) * jx - c23 * smu[4] + (smu[13] * jy + smu[15] * jz) * ir0;
  out[2] = (a + pyz + w) * jy - c23 * smu[6] + (smu[13] * jx + smu[14] * jz) * ir0;
  out[3] = (a + pyz - w) * jz - c23 * smu[8] + (smu[14] * jy + smu[15] * jx) * ir0;
}

template <class C>
__device__ __forceinline__ void meq_adjoint(D3Q15, const C (&smu)[15], C jx, C jy, C jz, C ir0,
                                            C (&out)[4]) {
  out[0] = -smu[1] + smu[2];
  const C a = (C(2) * smu[1] - C(10) * smu[2]) * ir0;    // e, eps: j^2, -5 j^2
  const C px = C(4) * smu[9] * ir0;                      // 3p_xx along j_x
  const C pyz = C(-2) * smu[9] * ir0;                    // 3p_xx along j_y, j_z
  const C w = C(2) * smu[10] * ir0;                      // p_ww along j_y (-w along j_z)
  const C c73 = C(7.0 / 3.0);
  out[1] = (a + px) * jx - c73 * smu[4] + (smu[11] * jy + smu[13] * jz) * ir0;
  out[2] = (a + pyz + w) * jy - c73 * smu[6] + (smu[11] * jx + smu[12] * jz) * ir0;
  out[3] = (a + pyz - w) * jz - c73 * smu[8] + (smu[12] * jy + smu[13] * jx) * ir0;
}

// One step back in time, one node per thread.  SMALL: node indices fit in 31 bits,
// so neighbour indices come from the node's wrapped coordinates in 32-bit
// arithmetic.
template <class L, class C, bool SMALL>
__global__ void __launch_bounds__(kAdjThreads, sizeof(C) == 4 ? LBM_ADJ_MINB_F32 : 3)
    adjoint_step_kernel(const SweepArgs<C> sa, AuxArgs a, AdjGeo ag, const C *__restrict__ f,
                        const C *__restrict__ lam_in, C *__restrict__ lam_out, double *gs_part) {
  constexpr int Q = L::Q;
  const long long N = a.N;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  C gsum[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) gsum[k] = C(0);
  const uint8_t cls = n < N ? a.cls[n] : (uint8_t)kSolid;
  if (cls != kSolid) {
    int x, y, z;
    {
      const long long r = n / a.nx;
      x = (int)(n - r * a.nx);
      y = (int)(r % a.ny);
      z = (int)(r / a.ny);
    }
    const C ir0 = sa.inv_rho0;
    C g[Q], lp[Q], lpre[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      g[i] = f[(long long)i * N + n];
      lpre[i] = C(0);
    }
    // advection transpose: lambda'_i(x) = lambda_i(x + e_i); solid entries of the
    // adjoint are kept at zero, so no class test is needed.  Neighbours follow the
    // periodic wrap, skewed along x by (sy, sz).
    const bool inside = x > 0 && x < a.nx - 1 && y > 0 && y < a.ny - 1 &&
                        (L::D == 2 || (z > 0 && z < a.nz - 1));
    if (inside) {
      // away from the faces of the box: a constant offset per direction
      const long long sx = a.nx, sxy = (long long)a.nx * a.ny;
      const C *base = lam_in + n;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        long long o = (long long)i * N;
        if (L::ex(i)) o += L::ex(i);
        if (L::ey(i)) o += L::ey(i) > 0 ? sx : -sx;
        if (L::ez(i)) o += L::ez(i) > 0 ? sxy : -sxy;
        lp[i] = base[o];
      }
    } else if constexpr (SMALL) {
      const Neighbours<L, true> nb(x, y, z, a.nx, a.ny, a.nz, a.sy, a.sz);
#pragma unroll
      for (int i = 0; i < Q; ++i) lp[i] = lam_in[(long long)i * N + nb(i)];
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        lp[i] = lam_in[(long long)i * N + wrap_index(x, y, z, L::ex(i), L::ey(i), L::ez(i), a.nx,
                                                     a.ny, a.nz, a.sy, a.sz)];
    }
    // boundary transpose and link gradients (Eq. 2.13)
    if (cls == kBoundary) {
      C gp[Q];
      C drho;
      collide<L, C>(g, gp, sa, drho);
      const LinkCoef<C> *coef = static_cast<const LinkCoef<C> *>(sa.geo.coef);
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
          // deviations suffice: A' + B' + C' = 0 removes the w_i rho0 parts
          const LinkCoef<C> dc = static_cast<const LinkCoef<C> *>(ag.dcoef)[k];
          C *acc = static_cast<C *>(ag.acc) + 2 * (long long)k;
          acc[0] += av * sa.wfac;           // W and its derivatives carry the step's factor
          acc[1] += av * (dc.a * g[dd] + dc.bb * gp[i] + dc.c * gp[dd]);
        }
      }
    }
    // collision transpose in moment space
    // the factored transforms (fmoments, fmt): fewer operations than the pair form
    // (FP64: the FP64 pipe bounds the step, backward 5.60 -> 4.59 s at 128^3 x 2000;
    // FP32: 0.349 -> 0.340 s, the gradient's difference from FP64 unchanged at 3.06e-5)
    C m[Q], mu[Q];
    fmoments<C>(L{}, g, m);
    fmoments<C>(L{}, lp, mu);
    const C jx = m[3], jy = m[5], jz = L::D == 3 ? m[7] : C(0);
    C smu[Q], nu[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      if (Rows<L>::cons(k)) {
        smu[k] = C(0);
        mu[k] *= C(1.0 / row_norm2<L>(k));
        continue;
      }
      smu[k] = sa.sn[k] * mu[k];                                      // s_k (M lambda')_k / |M_k|^2
      mu[k] *= C(1.0 / row_norm2<L>(k));
      gsum[k] = mu[k] * (meq(L{}, k, m[0], jx, jy, jz, ir0) - m[k]);   // d m'_k/d s_k
      nu[k] = mu[k] - smu[k];                                         // (1 - s_k) mu_k
    }
    C dq[4];
    meq_adjoint(L{}, smu, jx, jy, jz, ir0, dq);
    nu[0] = mu[0] + dq[0];
    nu[3] = mu[3] + dq[1];
    nu[5] = mu[5] + dq[2];
    if (L::D == 3) nu[7] = mu[7] + dq[3];
    // lambda(t) = M^T nu + boundary terms
    C t[Q];
    fmt<true, C>(L{}, nu, t);
#pragma unroll
    for (int i = 0; i < Q; ++i) lam_out[(long long)i * N + n] = lpre[i] + t[i];
  }
  // dJ/ds: block sums in the compute type (FP64 arithmetic is slow on this GPU),
  // added in FP64 to this block's own partial record (no atomics)
  C v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = C(0);
#pragma unroll
  for (int k = 0; k < Q; ++k)
    if (!Rows<L>::cons(k)) v[nc_slot<L>(k)] = gsum[k];
  const C wsum = warp_sum16(v);
  __shared__ C sh[kAdjThreads / 32][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((lane & 1) == 0) sh[warp][lane >> 1] = wsum;
  __syncthreads();
  if (threadIdx.x < Q && !Rows<L>::cons(threadIdx.x)) {
    int slot = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (k == (int)threadIdx.x) slot = nc_slot<L>(k);
    C t = C(0);
    for (int w = 0; w < kAdjThreads / 32; ++w) t += sh[w][slot];
    gs_part[(long long)blockIdx.x * Q + threadIdx.x] += (double)t;
  }
}

// One forward step in the natural layout, for recomputing a segment (push form):
// every fluid node collides its pre-collision populations f(t) (fin) and sends
// f'_i to slot i of x + e_i in fout, which then holds f(t+1); the populations that
// arrive through a cut link come from the single-node scheme (Eqs. 2.10, 2.13)
// into the node's own slot.  Same arithmetic as the fused sweep, so the states
// agree with the forward run's; slots of solid nodes receive values nobody reads.
// Reads and writes Q values per node, against the sweep-with-save's three.
template <class L, class C, bool SMALL>
__global__ void __launch_bounds__(kAdjThreads, sizeof(C) == 4 ? 6 : 3)
    recompute_step_kernel(const SweepArgs<C> sa, AuxArgs a, const C *__restrict__ fin,
                          C *__restrict__ fout) {
  constexpr int Q = L::Q;
  const long long N = a.N;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  C g[Q], gp[Q];
  const uint8_t cls = a.cls[n];
  if (cls == kSolid) return;
  int x, y, z;
  {
    const long long r = n / a.nx;
    x = (int)(n - r * a.nx);
    y = (int)(r % a.ny);
    z = (int)(r / a.ny);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] = fin[(long long)i * N + n];
  C drho;
  collide<L, C>(g, gp, sa, drho);
  if (!(fabs(drho) < C(1e6))) atomicOr(sa.status, 1);
  const bool inside = x > 0 && x < a.nx - 1 && y > 0 && y < a.ny - 1 &&
                      (L::D == 2 || (z > 0 && z < a.nz - 1));
  if (inside) {
    const long long sx = a.nx, sxy = (long long)a.nx * a.ny;
    C *base = fout + n;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      long long o = (long long)i * N;
      if (L::ex(i)) o += L::ex(i);
      if (L::ey(i)) o += L::ey(i) > 0 ? sx : -sx;
      if (L::ez(i)) o += L::ez(i) > 0 ? sxy : -sxy;
      base[o] = gp[i];
    }
  } else if constexpr (SMALL) {
    const Neighbours<L, true> nb(x, y, z, a.nx, a.ny, a.nz, a.sy, a.sz);
#pragma unroll
    for (int i = 0; i < Q; ++i) fout[(long long)i * N + nb(i)] = gp[i];
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      fout[(long long)i * N + wrap_index(x, y, z, L::ex(i), L::ey(i), L::ez(i), a.nx, a.ny, a.nz,
                                         a.sy, a.sz)] = gp[i];
  }
  if (cls == kBoundary) {
    const LinkCoef<C> *coef = static_cast<const LinkCoef<C> *>(sa.geo.coef);
    const int bi = a.bidx[n];
    const uint32_t mask = a.bmask[bi];
    const int off = a.boff[bi];
#pragma unroll
    for (int dd = 1; dd < Q; ++dd) {
      if (mask & (1u << dd)) {
        const LinkCoef<C> c = coef[off + __popc(mask & ((1u << dd) - 1u))];
        const int i = L::opp(dd);
        fout[(long long)i * N + n] =
            sa.one_minus_b * g[i] + c.a * g[dd] + c.bb * gp[i] + c.c * gp[dd] + c.w * sa.wfac;
      }
    }
  }
}

// add the per-link sums of one segment to the FP64 totals and clear them
template <class C>
__global__ void link_flush_kernel(C *acc, double *tot, long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    tot[j] += (double)acc[j];
    acc[j] = C(0);
  }
}

// sum of the per-block partial records: grad_s[k] = sum_b part[b*Q + k]; block k
// sums row k with a fixed order (deterministic)
template <int Q>
__global__ void __launch_bounds__(256) gs_finish_kernel(const double *part, long long n_blocks,
                                                        double *grad_s) {
  const int k = blockIdx.x;
  double v = 0.0;
  for (long long b = threadIdx.x; b < n_blocks; b += blockDim.x) v += part[b * Q + k];
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad_s[k] = sh[0];
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
                                const SweepArgs<float> &a32, const AuxArgs &a, const void *dcoef,
                                void *link_acc, const void *f, const void *lam_in, void *lam_out,
                                double *gs_part, cudaStream_t st) {
  const AdjGeo ag{dcoef, link_acc};
  const unsigned blocks = (unsigned)adjoint_partial_blocks(a.N);
  const bool small = a.N < (1LL << 31);
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    auto go = [&](const auto &sa, auto sm) {
      using C = std::remove_cv_t<std::remove_reference_t<decltype(sa.inv_rho0)>>;
      adjoint_step_kernel<L, C, decltype(sm)::value><<<blocks, kAdjThreads, 0, st>>>(
          sa, a, ag, static_cast<const C *>(f), static_cast<const C *>(lam_in),
          static_cast<C *>(lam_out), gs_part);
    };
    if (precision == 0) {
      if (small) go(a64, std::true_type{});
      else go(a64, std::false_type{});
    } else {
      if (small) go(a32, std::true_type{});
      else go(a32, std::false_type{});
    }
    return cudaGetLastError();
  });
}

cudaError_t launch_recompute_step(int lattice, int precision, const SweepArgs<double> &a64,
                                  const SweepArgs<float> &a32, const AuxArgs &a, const void *fin,
                                  void *fout, cudaStream_t st) {
  const unsigned blocks = (unsigned)adjoint_partial_blocks(a.N);
  const bool small = a.N < (1LL << 31);
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    auto go = [&](const auto &sa, auto sm) {
      using C = std::remove_cv_t<std::remove_reference_t<decltype(sa.inv_rho0)>>;
      recompute_step_kernel<L, C, decltype(sm)::value><<<blocks, kAdjThreads, 0, st>>>(
          sa, a, static_cast<const C *>(fin), static_cast<C *>(fout));
    };
    if (precision == 0) {
      if (small) go(a64, std::true_type{});
      else go(a64, std::false_type{});
    } else {
      if (small) go(a32, std::true_type{});
      else go(a32, std::false_type{});
    }
    return cudaGetLastError();
  });
}

cudaError_t launch_link_flush(int precision, void *link_acc, double *tot, long long n,
                              cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  if (precision == 0)
    link_flush_kernel<double><<<blocks, 256, 0, st>>>(static_cast<double *>(link_acc), tot, n);
  else
    link_flush_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float *>(link_acc), tot, n);
  return cudaGetLastError();
}

long long adjoint_partial_blocks(long long N) { return (N + kAdjThreads - 1) / kAdjThreads; }

cudaError_t launch_adjoint_finish(int lattice, const double *gs_part, long long n_blocks,
                                  double *grad_s, cudaStream_t st) {
  if (lattice == 0) gs_finish_kernel<9><<<9, 256, 0, st>>>(gs_part, n_blocks, grad_s);
  else if (lattice == 2) gs_finish_kernel<15><<<15, 256, 0, st>>>(gs_part, n_blocks, grad_s);
  else gs_finish_kernel<19><<<19, 256, 0, st>>>(gs_part, n_blocks, grad_s);
  return cudaGetLastError();
}

}  // namespace lbm
