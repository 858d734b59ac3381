// sweep.cuh -- the fused collide / stream / boundary sweep (one time step).
//
// One thread owns one node.  Populations live in one array in SoA order
// (population i of node n at i*N + n, x fastest) and are updated in place with
// the AA pattern:
//   even step  node x reads slot i of x, writes f'_i to slot opp(i) of x;
//   odd step   node x reads slot opp(i) of x - e_i, writes f'_i to slot i of x + e_i.
// Each node reads exactly the slots it writes, so a step needs one array and no
// synchronisation between threads.
//
// Cut links (Sec. 2 of arXiv:1712.08288).  For a fluid node x_f whose neighbour
// x_f + e_d is solid, the population i = opp(d) that would arrive from that
// neighbour is produced by the single-node scheme, Eqs. 2.10 and 2.13, from the
// node's own pre-collision f_i, f_d and post-collision f'_i, f'_d, which all sit in
// registers at that point.  The value is written where the next step looks for
// f_i(x_f, t+1): after an even step that is slot d of the solid neighbour
// x_f + e_d (a ghost slot no other node writes), after an odd step slot i of x_f
// itself (which only the solid node would otherwise write).  So the boundary
// costs no extra population traffic.
//
// Collision (Appendix, MRT): in deviation variables g = f - w rho0,
//   m = M g, m'_k = m_k - s_k (m_k - m^eq_k) for the non-conserved rows,
//   g' = g - M^-1 (m - m') + M^-1 (rho0 g_force at the j rows),
// with M^-1 = M^T diag(1/|M_k|^2) (rows of M are orthogonal).  Rows are either
// even or odd under e -> -e, so the products run over the sums s_p = g_i + g_ib
// and differences a_p = g_i - g_ib of opposite pairs.
#pragma once

#include "common.cuh"

namespace lbm {

// Equilibrium moments m^eq_k in deviation form (rho replaced by rho - rho0) for
// the incompressible equilibrium of Eq. 42, j = rho0 u.  These are the closed forms
// of M f^eq for the two moment bases (Lallemand & Luo 2000 for D2Q9; d'Humieres
// et al. 2002 for D3Q19 with w_eps = 3, w_epsj = -11/2, w_xx = -1/2).
template <class C>
__device__ __forceinline__ C meq(D2Q9, int k, C drho, C jx, C jy, C, C ir0) {
  switch (k) {
    case 1: return C(-2) * drho + C(3) * (jx * jx + jy * jy) * ir0;
    case 2: return drho - C(3) * (jx * jx + jy * jy) * ir0;
    case 4: return -jx;
    case 6: return -jy;
    case 7: return (jx * jx - jy * jy) * ir0;
    case 8: return jx * jy * ir0;
    default: return C(0);
  }
}
template <class C>
__device__ __forceinline__ C meq(D3Q19, int k, C drho, C jx, C jy, C jz, C ir0) {
  const C j2 = (jx * jx + jy * jy + jz * jz) * ir0;
  switch (k) {
    case 1: return C(-11) * drho + C(19) * j2;
    case 2: return C(3) * drho - C(5.5) * j2;
    case 4: return C(-2.0 / 3.0) * jx;
    case 6: return C(-2.0 / 3.0) * jy;
    case 8: return C(-2.0 / 3.0) * jz;
    case 9: return C(3) * jx * jx * ir0 - j2;
    case 10: return C(-0.5) * (C(3) * jx * jx * ir0 - j2);
    case 11: return (jy * jy - jz * jz) * ir0;
    case 12: return C(-0.5) * (jy * jy - jz * jz) * ir0;
    case 13: return jx * jy * ir0;
    case 14: return jy * jz * ir0;
    case 15: return jx * jz * ir0;
    default: return C(0);
  }
}

// compile-time row properties
template <class L>
constexpr unsigned odd_row_mask() {
  unsigned m = 0;
  for (int k = 0; k < L::Q; ++k)
    if (row_is_odd<L>(k)) m |= 1u << k;
  return m;
}
template <class L>
constexpr unsigned conserved_row_mask() {
  unsigned m = 0;
  for (int k = 0; k < L::Q; ++k)
    if (L::conserved(k)) m |= 1u << k;
  return m;
}
template <class L>
struct Rows {
  static constexpr unsigned kOdd = odd_row_mask<L>();
  static constexpr unsigned kConserved = conserved_row_mask<L>();
  static __device__ __forceinline__ constexpr bool odd(int k) { return (kOdd >> k) & 1u; }
  static __device__ __forceinline__ constexpr bool cons(int k) { return (kConserved >> k) & 1u; }
};

// acc + m * v with m an integer literal after unrolling (0 and +-1 fold away)
template <class C>
__device__ __forceinline__ C madd(C acc, int m, C v) {
  if (m == 0) return acc;
  if (m == 1) return acc + v;
  if (m == -1) return acc - v;
  return acc + C(m) * v;
}

// MRT collision with the body force, deviation variables, g -> gp.
template <class L, class C>
__device__ __forceinline__ void collide(const C (&g)[L::Q], C (&gp)[L::Q], const SweepArgs<C> &a,
                                        C &drho_out) {
  constexpr int Q = L::Q;
  constexpr int NP = L::NP;
  C s[NP], d[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = L::pair_first(p), ib = L::opp(i);
    s[p] = g[i] + g[ib];
    d[p] = g[i] - g[ib];
  }
  // conserved moments
  C drho = g[0];
#pragma unroll
  for (int p = 0; p < NP; ++p) drho += s[p];
  C jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = L::pair_first(p);
    jx = madd(jx, L::ex(i), d[p]);
    jy = madd(jy, L::ey(i), d[p]);
    jz = madd(jz, L::ez(i), d[p]);
  }
  drho_out = drho;
  const C ir0 = a.inv_rho0;
  // relaxed non-equilibrium parts r_k = s_k (m_k - m^eq_k) / |M_k|^2
  C r[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    if (Rows<L>::cons(k)) {
      r[k] = C(0);
      continue;
    }
    C m = C(0);
    if (Rows<L>::odd(k)) {
#pragma unroll
      for (int p = 0; p < NP; ++p) m = madd(m, L::M(k, L::pair_first(p)), d[p]);
    } else {
      m = madd(m, L::M(k, 0), g[0]);
#pragma unroll
      for (int p = 0; p < NP; ++p) m = madd(m, L::M(k, L::pair_first(p)), s[p]);
    }
    r[k] = a.sn[k] * (m - meq(L{}, k, drho, jx, jy, jz, ir0));
  }
  // back-transform of the change: g' = g - sum_k M(k, i) r_k + force
  {
    C e0 = C(0);
#pragma unroll
    for (int k = 0; k < Q; ++k)
      if (!Rows<L>::cons(k) && !Rows<L>::odd(k)) e0 = madd(e0, L::M(k, 0), r[k]);
    gp[0] = g[0] - e0;
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int i = L::pair_first(p), ib = L::opp(i);
    C ev = C(0), od = C(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      if (Rows<L>::cons(k)) continue;
      if (Rows<L>::odd(k)) od = madd(od, L::M(k, i), r[k]);
      else ev = madd(ev, L::M(k, i), r[k]);
    }
    C fi = C(0);
    fi = madd(fi, L::ex(i), a.F[0]);
    fi = madd(fi, L::ey(i), a.F[1]);
    if (L::D == 3) fi = madd(fi, L::ez(i), a.F[2]);
    const C odd_part = od - fi;
    gp[i] = g[i] - ev - odd_part;
    gp[ib] = g[ib] - ev + odd_part;
  }
}

template <class L, class T, bool ODD>
__global__ void __launch_bounds__(128) sweep_kernel(const SweepArgs<typename Storage<T>::C> a) {
  using C = typename Storage<T>::C;
  constexpr int Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long N = a.N;
  const long long n = x + (long long)a.nx * (y + (long long)a.ny * z);
  const uint8_t cls = __ldg(a.geo.cls + n);
  if (cls == kSolid) return;
  T *__restrict__ pop = static_cast<T *>(a.pop);
  const bool interior = x > 0 && x < a.nx - 1 && y > 0 && y < a.ny - 1 &&
                        (L::D == 2 || (z > 0 && z < a.nz - 1));
  const long long sx = 1, syy = a.nx, szz = (long long)a.nx * a.ny;

  C g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long src;
    if (!ODD) {
      src = (long long)i * N + n;
    } else {
      const long long nb =
          interior ? n - (L::ex(i) * sx + L::ey(i) * syy + L::ez(i) * szz)
                   : wrap_index(x, y, z, -L::ex(i), -L::ey(i), -L::ez(i), a.nx, a.ny, a.nz, a.sy,
                                a.sz);
      src = (long long)L::opp(i) * N + nb;
    }
    g[i] = Storage<T>::load(pop + src);
  }

  C gp[Q];
  C drho;
  collide<L, C>(g, gp, a, drho);
  if (!(fabs(drho) < C(1e6))) atomicOr(a.status, 1);

  // stream
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    long long dst;
    if (!ODD) {
      dst = (long long)L::opp(i) * N + n;
    } else {
      const long long nb =
          interior ? n + (L::ex(i) * sx + L::ey(i) * syy + L::ez(i) * szz)
                   : wrap_index(x, y, z, L::ex(i), L::ey(i), L::ez(i), a.nx, a.ny, a.nz, a.sy,
                                a.sz);
      dst = (long long)i * N + nb;
    }
    Storage<T>::store(pop + dst, gp[i]);
  }

  // single-node boundary scheme on the cut links of this node (Eqs. 2.10, 2.13)
  if (cls == kBoundary) {
    const int b = __ldg(a.geo.bidx + n);
    const uint32_t mask = __ldg(a.geo.bmask + b);
    const int off = __ldg(a.geo.boff + b);
    const LinkCoef<C> *coef = static_cast<const LinkCoef<C> *>(a.geo.coef);
#pragma unroll
    for (int dd = 1; dd < Q; ++dd) {
      if (mask & (1u << dd)) {
        const LinkCoef<C> c = coef[off + __popc(mask & ((1u << dd) - 1u))];
        const int i = L::opp(dd);
        const C v = a.one_minus_b * g[i] + c.a * g[dd] + c.bb * gp[i] + c.c * gp[dd] + c.w;
        long long dst;
        if (!ODD) {
          // slot dd of the solid neighbour x_f + e_dd
          const long long nb =
              interior ? n + (L::ex(dd) * sx + L::ey(dd) * syy + L::ez(dd) * szz)
                       : wrap_index(x, y, z, L::ex(dd), L::ey(dd), L::ez(dd), a.nx, a.ny, a.nz,
                                    a.sy, a.sz);
          dst = (long long)dd * N + nb;
        } else {
          dst = (long long)i * N + n;
        }
        Storage<T>::store(pop + dst, v);
      }
    }
  }
}

template <class L, class T>
cudaError_t launch_sweep_t(bool odd, const SweepArgs<typename Storage<T>::C> &a, cudaStream_t st) {
  const int bx = a.nx >= 128 ? 128 : (a.nx >= 64 ? 64 : 32);
  dim3 block(bx, 1, 1);
  dim3 grid((a.nx + bx - 1) / bx, a.ny, a.nz);
  if (odd) sweep_kernel<L, T, true><<<grid, block, 0, st>>>(a);
  else sweep_kernel<L, T, false><<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lbm
