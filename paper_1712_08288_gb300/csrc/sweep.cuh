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
// registers at that point.  The value goes where the next step looks for
// f_i(x_f, t+1): after an odd step into slot i of x_f itself (which only the solid
// node would otherwise write); after an even step into the link's entry of a
// compact link buffer, which the next odd step reads in place of slot d of the
// solid neighbour.  Solid nodes' slots are never written.
//
// Collision (Appendix, MRT): in deviation variables g = f - w rho0,
//   m = M g, m'_k = m_k - s_k (m_k - m^eq_k) for the non-conserved rows,
//   g' = g - M^-1 (m - m') + M^-1 (rho0 g_force at the j rows),
// with M^-1 = M^T diag(1/|M_k|^2) (rows of M are orthogonal).  Rows are either
// even or odd under e -> -e, so the products run over the sums s_p = g_i + g_ib
// and differences a_p = g_i - g_ib of opposite pairs.
#pragma once

#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace lbm {

// Equilibrium moments m^eq_k in deviation form (rho replaced by rho - rho0) for
// the incompressible equilibrium of Eq. 42, j = rho0 u.  These are the closed forms
// of M f^eq for the moment bases (Lallemand & Luo 2000 for D2Q9; d'Humieres et
// al. 2002 for D3Q19 with w_eps = 3, w_epsj = -11/2, w_xx = -1/2; the Appendix's
// D3Q15 basis below).
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

// D3Q15 (Appendix basis): e^eq = -rho + j^2/rho0, eps^eq = rho - 5 j^2/rho0,
// q^eq = -7/3 j, second-order rows j_a j_b / rho0 combinations, m_xyz^eq = 0
template <class C>
__device__ __forceinline__ C meq(D3Q15, int k, C drho, C jx, C jy, C jz, C ir0) {
  const C j2 = (jx * jx + jy * jy + jz * jz) * ir0;
  switch (k) {
    case 1: return -drho + j2;
    case 2: return drho - C(5) * j2;
    case 4: return C(-7.0 / 3.0) * jx;
    case 6: return C(-7.0 / 3.0) * jy;
    case 8: return C(-7.0 / 3.0) * jz;
    case 9: return C(3) * jx * jx * ir0 - j2;
    case 10: return (jy * jy - jz * jz) * ir0;
    case 11: return jx * jy * ir0;
    case 12: return jy * jz * ir0;
    case 13: return jx * jz * ir0;
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

// D3Q19 collision with the moment sums and the back-transform factored by hand: the
// rows of M share partial sums over the face pairs, the edge pairs of each plane and
// all edges (rho, e, eps from the face and edge sums; the second-order rows from the
// three plane sums; q_a = j_a - 5 d_a), and the back-transform shares the common
// edge and face parts and the plane parts.  Same operator as the generic pair form
// below, with about a third fewer operations; rounding order differs.
template <class C>
__device__ __forceinline__ void collide_d3q19(const C (&g)[19], C (&gp)[19], const SweepArgs<C> &a,
                                              C &drho_out) {
  C s[9], d[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    s[p] = g[2 * p + 1] + g[2 * p + 2];
    d[p] = g[2 * p + 1] - g[2 * p + 2];
  }
  const C F = s[0] + s[1] + s[2];
  const C Exy = s[3] + s[4], Exz = s[5] + s[6], Eyz = s[7] + s[8];
  const C E = Exy + Exz + Eyz;
  const C drho = g[0] + F + E;
  const C jx = d[0] + d[3] + d[4] + d[5] + d[6];
  const C jy = d[1] + d[3] - d[4] + d[7] + d[8];
  const C jz = d[2] + d[5] - d[6] + d[7] - d[8];
  drho_out = drho;
  const C ir0 = a.inv_rho0;
  const C Exyz = Exy + Exz - C(2) * Eyz;
  C m[19];
  m[1] = C(-30) * g[0] - C(11) * F + C(8) * E;
  m[2] = C(12) * g[0] - C(4) * F + E;
  m[4] = jx - C(5) * d[0];
  m[6] = jy - C(5) * d[1];
  m[8] = jz - C(5) * d[2];
  m[9] = C(2) * s[0] - s[1] - s[2] + Exyz;
  m[10] = C(-4) * s[0] + C(2) * (s[1] + s[2]) + Exyz;
  m[11] = s[1] - s[2] + Exy - Exz;
  m[12] = C(2) * (s[2] - s[1]) + Exy - Exz;
  m[13] = s[3] - s[4];
  m[14] = s[7] - s[8];
  m[15] = s[5] - s[6];
  m[16] = d[3] + d[4] - d[5] - d[6];
  m[17] = d[4] - d[3] + d[7] + d[8];
  m[18] = d[5] - d[6] - d[7] + d[8];
  C r[19];
#pragma unroll
  for (int k = 1; k < 19; ++k)
    if (!D3Q19::conserved(k)) r[k] = a.sn[k] * (m[k] - meq(D3Q19{}, k, drho, jx, jy, jz, ir0));
  // back-transform: even parts per pair from shared face / edge / plane terms
  const C Cf = C(-11) * r[1] - C(4) * r[2], Ce = C(8) * r[1] + r[2];
  const C A = r[9] + r[10], B = r[11] + r[12];
  const C Y = Cf - r[9] + C(2) * r[10], Z = r[11] - C(2) * r[12];
  const C Pxy = Ce + A + B, Pxz = Ce + A - B, Pyz = Ce - C(2) * A;
  C ev[9], od[9];
  ev[0] = Cf + C(2) * r[9] - C(4) * r[10];
  ev[1] = Y + Z;
  ev[2] = Y - Z;
  ev[3] = Pxy + r[13];
  ev[4] = Pxy - r[13];
  ev[5] = Pxz + r[15];
  ev[6] = Pxz - r[15];
  ev[7] = Pyz + r[14];
  ev[8] = Pyz - r[14];
  // odd parts minus the force term of the pair's first direction: with the force
  // folded into the flux rates (ra = r_a - F_a) the edge pairs share the sums
  // (ra + r16), (rb - r17), ... of their two directions
  const C F0 = a.F[0], F1 = a.F[1], F2 = a.F[2];
  const C rx = r[4] - F0, ry = r[6] - F1, rz = r[8] - F2;
  od[0] = C(-4) * rx - C(5) * F0;
  od[1] = C(-4) * ry - C(5) * F1;
  od[2] = C(-4) * rz - C(5) * F2;
  const C xa = rx + r[16], ya = ry - r[17];
  od[3] = xa + ya;
  od[4] = xa - ya;
  const C xb = rx - r[16], zb = rz + r[18];
  od[5] = xb + zb;
  od[6] = xb - zb;
  const C yc = ry + r[17], zc = rz - r[18];
  od[7] = yc + zc;
  od[8] = yc - zc;
  gp[0] = g[0] - (C(-30) * r[1] + C(12) * r[2]);
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    gp[2 * p + 1] = g[2 * p + 1] - ev[p] - od[p];
    gp[2 * p + 2] = g[2 * p + 2] - ev[p] + od[p];
  }
}

// Factored moment transforms per lattice: m = M v (fmoments) and out = M^T nu (fmt)
// with the sums shared: pair sums s_p and differences d_p, the sums over faces,
// edges or corners (rho, e, eps), the plane sums (the second-order rows), the fluxes
// q_a from j_a and the face differences.  fmt<false> leaves out row 0 (rho), which a
// collision never relaxes.  factored_matches_M<L>() compares both with the lattice's M
// entry by entry; the static_asserts below run it at compile time.
template <class C>
LBM_HD constexpr void fmoments(D2Q9, const C (&v)[9], C (&m)[9]) {
  // pairs (1,3), (2,4) faces, (5,7), (6,8) diagonals
  const C s0 = v[1] + v[3], s1 = v[2] + v[4], s2 = v[5] + v[7], s3 = v[6] + v[8];
  const C d0 = v[1] - v[3], d1 = v[2] - v[4], d2 = v[5] - v[7], d3 = v[6] - v[8];
  const C F = s0 + s1, E = s2 + s3;
  const C jx = d0 + d2 - d3, jy = d1 + d2 + d3;
  m[0] = v[0] + F + E;
  m[1] = C(-4) * v[0] - F + C(2) * E;
  m[2] = C(4) * v[0] - C(2) * F + E;
  m[3] = jx;
  m[4] = jx - C(3) * d0;
  m[5] = jy;
  m[6] = jy - C(3) * d1;
  m[7] = s0 - s1;
  m[8] = s2 - s3;
}
template <bool kRho, class C>
LBM_HD constexpr void fmt(D2Q9, const C (&nu)[9], C (&out)[9]) {
  const C Cf = kRho ? nu[0] - nu[1] - C(2) * nu[2] : -nu[1] - C(2) * nu[2];
  const C Ce = kRho ? nu[0] + C(2) * nu[1] + nu[2] : C(2) * nu[1] + nu[2];
  const C X = nu[3] + nu[4], Y = nu[5] + nu[6];
  const C ev0 = Cf + nu[7], ev1 = Cf - nu[7], ev2 = Ce + nu[8], ev3 = Ce - nu[8];
  const C od0 = nu[3] - C(2) * nu[4], od1 = nu[5] - C(2) * nu[6], od2 = X + Y, od3 = Y - X;
  out[0] = kRho ? nu[0] - C(4) * nu[1] + C(4) * nu[2] : C(-4) * nu[1] + C(4) * nu[2];
  out[1] = ev0 + od0;
  out[3] = ev0 - od0;
  out[2] = ev1 + od1;
  out[4] = ev1 - od1;
  out[5] = ev2 + od2;
  out[7] = ev2 - od2;
  out[6] = ev3 + od3;
  out[8] = ev3 - od3;
}

template <class C>
LBM_HD constexpr void fmoments(D3Q15, const C (&v)[15], C (&m)[15]) {
  // pairs (1,2), (3,4), (5,6) faces, (7,14), (8,13), (9,12), (10,11) corners
  const C s0 = v[1] + v[2], s1 = v[3] + v[4], s2 = v[5] + v[6];
  const C d0 = v[1] - v[2], d1 = v[3] - v[4], d2 = v[5] - v[6];
  const C s3 = v[7] + v[14], s4 = v[8] + v[13], s5 = v[9] + v[12], s6 = v[10] + v[11];
  const C d3 = v[7] - v[14], d4 = v[8] - v[13], d5 = v[9] - v[12], d6 = v[10] - v[11];
  const C F = s0 + s1 + s2;
  const C ca = s3 + s6, cb = s4 + s5, cc = s3 - s6, cd = s4 - s5;
  const C ce = d3 + d6, cf = d4 + d5, cg = d3 - d6, ch = d4 - d5;
  const C K = ca + cb;
  const C jx = d0 + cg - ch, jy = d1 + cg + ch, jz = d2 + ce + cf;
  m[0] = v[0] + F + K;
  m[1] = C(-2) * v[0] - F + K;
  m[2] = C(16) * v[0] - C(4) * F + K;
  m[3] = jx;
  m[4] = jx - C(5) * d0;
  m[5] = jy;
  m[6] = jy - C(5) * d1;
  m[7] = jz;
  m[8] = jz - C(5) * d2;
  m[9] = C(2) * s0 - s1 - s2;
  m[10] = s1 - s2;
  m[11] = ca - cb;
  m[12] = cc + cd;
  m[13] = cc - cd;
  m[14] = ce - cf;
}
template <bool kRho, class C>
LBM_HD constexpr void fmt(D3Q15, const C (&nu)[15], C (&out)[15]) {
  const C Cf = kRho ? nu[0] - nu[1] - C(4) * nu[2] : -nu[1] - C(4) * nu[2];
  const C Cc = kRho ? nu[0] + nu[1] + nu[2] : nu[1] + nu[2];
  const C ev0 = Cf + C(2) * nu[9], ev1 = Cf - nu[9] + nu[10], ev2 = Cf - nu[9] - nu[10];
  const C od0 = nu[3] - C(4) * nu[4], od1 = nu[5] - C(4) * nu[6], od2 = nu[7] - C(4) * nu[8];
  const C P = Cc + nu[12], Qm = Cc - nu[12], A = nu[11] + nu[13], B = nu[11] - nu[13];
  const C X = nu[3] + nu[4], Y = nu[5] + nu[6], Z = nu[7] + nu[8];
  const C YZp = Y + Z, YZm = Z - Y, Xp = X + nu[14], Xm = X - nu[14];
  out[0] = kRho ? nu[0] - C(2) * nu[1] + C(16) * nu[2] : C(-2) * nu[1] + C(16) * nu[2];
  out[1] = ev0 + od0;
  out[2] = ev0 - od0;
  out[3] = ev1 + od1;
  out[4] = ev1 - od1;
  out[5] = ev2 + od2;
  out[6] = ev2 - od2;
  out[7] = (P + A) + (YZp + Xp);
  out[14] = (P + A) - (YZp + Xp);
  out[8] = (P - A) + (YZp - Xp);
  out[13] = (P - A) - (YZp - Xp);
  out[9] = (Qm - B) + (YZm + Xm);
  out[12] = (Qm - B) - (YZm + Xm);
  out[10] = (Qm + B) + (YZm - Xm);
  out[11] = (Qm + B) - (YZm - Xm);
}

template <class C>
LBM_HD constexpr void fmoments(D3Q19, const C (&v)[19], C (&m)[19]) {
  // pairs (2p+1, 2p+2): faces p = 0..2, edges p = 3..8 (xy, xy, xz, xz, yz, yz)
  C s[9] = {}, d[9] = {};
  for (int p = 0; p < 9; ++p) {
    s[p] = v[2 * p + 1] + v[2 * p + 2];
    d[p] = v[2 * p + 1] - v[2 * p + 2];
  }
  const C F = s[0] + s[1] + s[2];
  const C Exy = s[3] + s[4], Exz = s[5] + s[6], Eyz = s[7] + s[8];
  const C E = Exy + Exz + Eyz;
  const C jx = d[0] + d[3] + d[4] + d[5] + d[6];
  const C jy = d[1] + d[3] - d[4] + d[7] + d[8];
  const C jz = d[2] + d[5] - d[6] + d[7] - d[8];
  const C Exyz = Exy + Exz - C(2) * Eyz;
  const C Wxy = Exy - Exz;
  m[0] = v[0] + F + E;
  m[1] = C(-30) * v[0] - C(11) * F + C(8) * E;
  m[2] = C(12) * v[0] - C(4) * F + E;
  m[3] = jx;
  m[4] = jx - C(5) * d[0];
  m[5] = jy;
  m[6] = jy - C(5) * d[1];
  m[7] = jz;
  m[8] = jz - C(5) * d[2];
  m[9] = C(2) * s[0] - s[1] - s[2] + Exyz;
  m[10] = C(-4) * s[0] + C(2) * (s[1] + s[2]) + Exyz;
  m[11] = s[1] - s[2] + Wxy;
  m[12] = C(2) * (s[2] - s[1]) + Wxy;
  m[13] = s[3] - s[4];
  m[14] = s[7] - s[8];
  m[15] = s[5] - s[6];
  m[16] = d[3] + d[4] - d[5] - d[6];
  m[17] = d[4] - d[3] + d[7] + d[8];
  m[18] = d[5] - d[6] - d[7] + d[8];
}
template <bool kRho, class C>
LBM_HD constexpr void fmt(D3Q19, const C (&nu)[19], C (&out)[19]) {
  // even parts per pair: rows rho, e, eps (faces Cf, edges Ce) and the plane rows
  const C Cf = kRho ? nu[0] - C(11) * nu[1] - C(4) * nu[2] : C(-11) * nu[1] - C(4) * nu[2];
  const C Ce = kRho ? nu[0] + C(8) * nu[1] + nu[2] : C(8) * nu[1] + nu[2];
  const C A = nu[9] + nu[10], B = nu[11] + nu[12];
  const C Y = Cf - nu[9] + C(2) * nu[10], Z = nu[11] - C(2) * nu[12];
  const C Pxy = Ce + A + B, Pxz = Ce + A - B, Pyz = Ce - C(2) * A;
  C ev[9] = {}, od[9] = {};
  ev[0] = Cf + C(2) * nu[9] - C(4) * nu[10];
  ev[1] = Y + Z;
  ev[2] = Y - Z;
  ev[3] = Pxy + nu[13];
  ev[4] = Pxy - nu[13];
  ev[5] = Pxz + nu[15];
  ev[6] = Pxz - nu[15];
  ev[7] = Pyz + nu[14];
  ev[8] = Pyz - nu[14];
  // odd parts: j_a and q_a rows (faces: j_a - 4 q_a, edges: j_a + q_a) and m_x,y,z
  od[0] = nu[3] - C(4) * nu[4];
  od[1] = nu[5] - C(4) * nu[6];
  od[2] = nu[7] - C(4) * nu[8];
  const C rx = nu[3] + nu[4], ry = nu[5] + nu[6], rz = nu[7] + nu[8];
  const C xa = rx + nu[16], ya = ry - nu[17];
  od[3] = xa + ya;
  od[4] = xa - ya;
  const C xb = rx - nu[16], zb = rz + nu[18];
  od[5] = xb + zb;
  od[6] = xb - zb;
  const C yc = ry + nu[17], zc = rz - nu[18];
  od[7] = yc + zc;
  od[8] = yc - zc;
  out[0] = kRho ? nu[0] - C(30) * nu[1] + C(12) * nu[2] : C(-30) * nu[1] + C(12) * nu[2];
  for (int p = 0; p < 9; ++p) {
    out[2 * p + 1] = ev[p] + od[p];
    out[2 * p + 2] = ev[p] - od[p];
  }
}

template <class L>
constexpr bool factored_matches_M() {
  constexpr int Q = L::Q;
  for (int i = 0; i < Q; ++i) {
    int v[Q] = {}, m[Q] = {};
    v[i] = 1;
    fmoments<int>(L{}, v, m);
    for (int k = 0; k < Q; ++k)
      if (m[k] != L::M(k, i)) return false;
  }
  for (int k = 0; k < Q; ++k) {
    int nu[Q] = {}, out[Q] = {}, out0[Q] = {};
    nu[k] = 1;
    fmt<true, int>(L{}, nu, out);
    fmt<false, int>(L{}, nu, out0);
    for (int i = 0; i < Q; ++i) {
      if (out[i] != L::M(k, i)) return false;
      if (out0[i] != (k == 0 ? 0 : L::M(k, i))) return false;
    }
  }
  return true;
}
static_assert(factored_matches_M<D2Q9>(), "factored D2Q9 transforms differ from M");
static_assert(factored_matches_M<D3Q15>(), "factored D3Q15 transforms differ from M");
static_assert(factored_matches_M<D3Q19>(), "factored D3Q19 transforms differ from M");

// MRT collision through the factored transforms (D2Q9, D3Q15): r_k = s_k (m_k - m^eq_k)
// / |M_k|^2 on the relaxed rows, r = -F on the momentum rows (the force term), and
// g' = g - M^T r.
template <class L, class C>
__device__ __forceinline__ void collide_factored(const C (&g)[L::Q], C (&gp)[L::Q], const SweepArgs<C> &a,
                                                 C &drho_out) {
  constexpr int Q = L::Q;
  C m[Q];
  fmoments<C>(L{}, g, m);
  const C drho = m[0], jx = m[3], jy = m[5], jz = L::D == 3 ? m[7] : C(0);
  drho_out = drho;
  const C ir0 = a.inv_rho0;
  C r[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k)
    r[k] = Rows<L>::cons(k) ? C(0) : a.sn[k] * (m[k] - meq(L{}, k, drho, jx, jy, jz, ir0));
  r[3] = -a.F[0];
  r[5] = -a.F[1];
  if constexpr (L::D == 3) r[7] = -a.F[2];
  C t[Q];
  fmt<false, C>(L{}, r, t);
#pragma unroll
  for (int i = 0; i < Q; ++i) gp[i] = g[i] - t[i];
}

// MRT collision with the body force, deviation variables, g -> gp.  T is the
// storage type (it selects the form of the D3Q19 collision).
template <class L, class C, class T = C>
__device__ __forceinline__ void collide(const C (&g)[L::Q], C (&gp)[L::Q], const SweepArgs<C> &a,
                                        C &drho_out) {
  if constexpr (std::is_same_v<L, D3Q19> && (sizeof(C) == 8 || sizeof(T) == 2)) {
    // The factored form where the sweep is bound by instruction issue: FP64 (the FP64
    // pipe; 22 % faster) and 16-bit storage (half the bytes of FP32, the same
    // instructions; 8 % faster).  FP32 storage is bound by memory traffic, runs at
    // the same speed with either form, and keeps the generic form, whose rounding
    // tracks FP64 closer (E_r 0.2 % from FP64 after 20000 steps, against 2.3 % with
    // the factored form).
    collide_d3q19<C>(g, gp, a, drho_out);
    return;
  } else if constexpr (!std::is_same_v<L, D3Q19> && (sizeof(C) == 8 || sizeof(T) == 2)) {
    // D2Q9 and D3Q15 likewise
    collide_factored<L, C>(g, gp, a, drho_out);
    return;
  }
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

// Wrap an index that is at most one period outside [0, n).
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Linear index of the neighbour x + e_k (periodic, x-wrap skewed by (sy, sz) when
// SKEW).  The per-node part (wrapped x +- 1 and the skew-shifted rows) is computed
// once; per direction, row coordinates are wrapped only where that direction can
// leave the range, which the compiler resolves at compile time.
template <class L, bool SKEW>
struct Neighbours {
  int x, y, z, xm, xp, ym, yp, zm, zp, nx, ny, nz;
  __device__ __forceinline__ Neighbours(int x_, int y_, int z_, int nx_, int ny_, int nz_, int sy,
                                        int sz)
      : x(x_), y(y_), z(z_), nx(nx_), ny(ny_), nz(nz_) {
    xm = x - 1;
    xp = x + 1;
    const bool cm = xm < 0, cp = xp >= nx;
    if (cm) xm += nx;
    if (cp) xp -= nx;
    ym = yp = y;
    zm = zp = z;
    if (SKEW) {
      // crossing x = 0 downward lands at (nx-1, y+sy, z+sz); crossing x = nx-1 upward
      // lands at (0, y-sy, z-sz) (the field is invariant under (nx, sy, sz))
      if (cm) { ym += sy; zm += sz; }
      if (cp) { yp -= sy; zp -= sz; }
    }
  }
  __device__ __forceinline__ int operator()(int k) const {
    const int ex = L::ex(k), ey = L::ey(k), ez = L::ez(k);
    const int xx = ex < 0 ? xm : (ex > 0 ? xp : x);
    int yy = (ex < 0 ? ym : (ex > 0 ? yp : y)) + ey;
    if (ey != 0 || (SKEW && ex != 0)) yy = wrap1(yy, ny);
    int zz = 0;
    if (L::D == 3) {
      zz = (ex < 0 ? zm : (ex > 0 ? zp : z)) + ez;
      if (ez != 0 || (SKEW && ex != 0)) zz = wrap1(zz, nz);
    }
    return xx + nx * (yy + ny * zz);
  }
};

// ---------------------------------------------------------------------------
// Bulk-copy pipeline helpers (inline PTX, sm_90+): mbarrier with transaction
// count, cp.async.bulk global -> shared.
// ---------------------------------------------------------------------------
constexpr uint32_t kSuspendHintNs = 1000000;   // 1 ms upper bound per poll
constexpr int kWaitLimit = kWaitLimitDefault;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// try_wait with a suspend-time hint: a thread whose phase has not completed sleeps
// (up to the hint) instead of spinning, so waiting warps do not take issue slots
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return done != 0;
}
// bounded wait: gives up after `polls` polls, each suspending for at most
// kSuspendHintNs; the default kWaitLimit polls is about 1 s, far beyond any
// legitimate copy latency
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  int polls = kWaitLimit) {
  for (int it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Work decomposition.  A tile is a run of TW nodes along x (TW = kTileW = 64, or
// 32-node half tiles: the single-context FP64 sweep and, by choice, batches) that
// holds at least one fluid node; tiles are listed once per geometry.  A warp processes a tile TW/32 nodes per lane, one
// node after the other.  Every warp owns a private pipeline of kStages shared-memory
// stages: stage s holds the Q population row windows of one tile (each window up to
// TW + 16/sizeof(T) elements, start aligned down to 16 bytes), filled by bulk copies
// that complete on the warp's own mbarrier.  32-node tiles take more stages with 4-
// and 2-byte storage (3 and 5): a warp keeps most of its bytes in flight while a
// block still fits the shared memory of the 64-node layout.  FP64 storage keeps 2
// stages in 32-node tiles: its sweep is bound by the FP64 pipe, and half the shared
// memory doubles the blocks per SM (4 instead of 2).  Warps never wait for each other.
constexpr int kWarpsPerBlock = 4;

#ifndef LBM_STAGES_4B
#define LBM_STAGES_4B 2
#endif
#ifndef LBM_STAGES_8B
#define LBM_STAGES_8B 2
#endif
#ifndef LBM_STAGES_8B_32
#define LBM_STAGES_8B_32 2
#endif
template <class T, int TW = kTileW>
struct StageShape {
  static_assert(TW == 32 || TW == 64, "tiles are one or two nodes per lane wide");
  static constexpr int kStages = TW == 64 ? (sizeof(T) == 8 ? LBM_STAGES_8B : (sizeof(T) == 4 ? LBM_STAGES_4B : 3))
                                          : (sizeof(T) == 2 ? 5 : (sizeof(T) == 8 ? LBM_STAGES_8B_32 : 3));
  static constexpr int kWidth = TW + 16 / (int)sizeof(T);   // elements per window
  static constexpr int kRecs = TW + 4;                       // record window (uint32)
};

// Byte layout of one stage: Q population windows, then the record window; after
// all stages, the barriers and the offsets (Q + 1 per stage).
template <class L, class T, int TW = kTileW>
struct StageLayout {
  using SS = StageShape<T, TW>;
  static constexpr size_t kPop = (size_t)L::Q * SS::kWidth * sizeof(T);
  static constexpr size_t kRec = kPop;
  static constexpr size_t kStage = (kRec + SS::kRecs * sizeof(uint32_t) + 15) / 16 * 16;
  static constexpr size_t kBars = SS::kStages * kStage;
  static constexpr size_t kOffs = kBars + SS::kStages * sizeof(uint64_t);
  static constexpr int kNOff = L::Q + 1;
};

// bytes of one warp's pipeline, a multiple of 128 so that every warp's stages
// start 128-byte aligned
template <class L, class T, int TW = kTileW>
__host__ __device__ constexpr size_t warp_smem_bytes() {
  using SL = StageLayout<L, T, TW>;
  return (SL::kOffs + StageShape<T, TW>::kStages * SL::kNOff * sizeof(int) + 127) / 128 * 128;
}
static_assert(warp_smem_bytes<D3Q19, float>() % 128 == 0, "warp region alignment");
static_assert(warp_smem_bytes<D3Q19, float, 32>() % 128 == 0, "warp region alignment");
static_assert(StageLayout<D3Q19, float, 32>::kRec % 16 == 0 && StageLayout<D3Q19, double, 32>::kRec % 16 == 0 &&
                  StageLayout<D3Q19, __half, 32>::kRec % 16 == 0 && StageLayout<D2Q9, __half, 32>::kRec % 16 == 0 &&
                  StageLayout<D3Q15, __half, 32>::kRec % 16 == 0 && StageLayout<D3Q15, __half>::kRec % 16 == 0,
              "record window alignment");
static_assert(StageLayout<D3Q19, float>::kRec % 16 == 0 && StageLayout<D3Q19, double>::kRec % 16 == 0 &&
                  StageLayout<D3Q19, __half>::kRec % 16 == 0 && StageLayout<D2Q9, __half>::kRec % 16 == 0,
              "record window alignment");
static_assert((StageShape<float>::kWidth * sizeof(float)) % 16 == 0, "window stride");
static_assert((StageShape<double>::kWidth * sizeof(double)) % 16 == 0, "window stride");
static_assert((StageShape<__half>::kWidth * sizeof(__half)) % 16 == 0, "window stride");

// aligned-down source of a window and the element offset of its first element
template <class E>
__device__ __forceinline__ const char *align16(const E *p, int &off_elems) {
  const char *pc = reinterpret_cast<const char *>(p);
  const char *pa = reinterpret_cast<const char *>(reinterpret_cast<uintptr_t>(pc) & ~(uintptr_t)15);
  off_elems = (int)((pc - pa) / (long long)sizeof(E));
  return pa;
}

// One warp fills one stage with everything a tile needs, lane i issuing copy i:
// lanes 0..Q-1 the population row windows (even step: window [x0, x0+TW) of slot
// i in the tile's own row; odd step: [x0 - ex_i, x0 - ex_i + TW) of slot opp(i)
// in row (y - ey_i, z - ez_i)), lane Q the tile's packed boundary records.  Every
// copy starts at the 16-byte boundary at or before its first element and covers its
// window rounded up to 16 bytes; off[] records where each first element landed.
// The offsets are stored before lane 0's arrive (release), so a lane that has
// waited on the barrier sees them.  All lanes call.
template <class L, class T, bool ODD, bool ALIGNED, class I, int TW>
__device__ __forceinline__ void issue_tile(const SweepArgs<typename Storage<T>::C> &a,
                                           const TileDesc &td, unsigned char *stage, int *off,
                                           uint64_t *bar) {
  using SL = StageLayout<L, T, TW>;
  constexpr int W = StageShape<T, TW>::kWidth;
  const int lane = threadIdx.x & 31;
  const int ty = td.yz & 0xffff, tz = td.yz >> 16;
  const char *src = nullptr, *src2 = nullptr;
  void *dst = nullptr, *dst2 = nullptr;
  uint32_t bytes = 0;
  if (lane < L::Q) {
    const int i = lane;
    int slot = i, yy = ty, zz = tz, xs = td.x0;
    if (ODD) {
      slot = L::opp_rt(i);
      yy = wrap1(ty - DirBits<L>::ey(i), a.ny);
      zz = (L::D == 3) ? wrap1(tz - DirBits<L>::ez(i), a.nz) : 0;
      xs = td.x0 - DirBits<L>::ex(i);
    }
    const T *pop = static_cast<const T *>(a.pop);
    const I elem = (I)slot * (I)a.S + (I)a.nx * ((I)yy + (I)a.ny * zz) + xs;
    int o;
    src = align16(pop + elem, o);
    off[i] = o;
    bytes = ((uint32_t)((o + TW) * (int)sizeof(T)) + 15u) & ~15u;
    dst = stage + (size_t)i * W * sizeof(T);
    if constexpr (ODD && ALIGNED) {
      // Windows that cross the periodic x-wrap (rows start on 16-byte boundaries):
      // the element read across x = 0 (column nx-1 of the row shifted by (+sy, +sz))
      // or across x = nx-1 (column 0 of the row shifted by (-sy, -sz)) comes from a
      // second 16-byte copy placed where the window expects it, and the main copy
      // stops at the row's end.
      constexpr int E16 = 16 / (int)sizeof(T);
      const int ex = DirBits<L>::ex(i);
      const bool lo = ex > 0 && td.x0 == 0;
      const bool hi = ex < 0 && td.x0 + TW > a.nx - 1;
      if (lo || hi) {
        const int sy = lo ? a.sy : -a.sy, sz = lo ? a.sz : -a.sz;
        const int yw = wrap1(yy + sy, a.ny);
        const int zw = (L::D == 3) ? wrap1(zz + sz, a.nz) : 0;
        const I rw = (I)slot * (I)a.S + (I)a.nx * ((I)yw + (I)a.ny * zw);
        if (lo) {
          // main copy: [0, TW) behind a 16-byte gap; chunk [nx-E16, nx) in the gap
          src = reinterpret_cast<const char *>(pop + elem + 1);
          dst = stage + ((size_t)i * W + E16) * sizeof(T);
          bytes = TW * sizeof(T);
          src2 = reinterpret_cast<const char *>(pop + rw + (a.nx - E16));
          dst2 = stage + (size_t)i * W * sizeof(T);
        } else {
          // main copy: [x0, nx); chunk [0, E16) of the wrapped row right after it
          bytes = (uint32_t)((a.nx - td.x0) * (int)sizeof(T));
          src2 = reinterpret_cast<const char *>(pop + rw);
          dst2 = stage + ((size_t)i * W + (a.nx - td.x0)) * sizeof(T);
        }
      }
    }
  } else if (lane == L::Q) {
    const int nrec = __popcll(td.bnd);
    int o;
    src = align16(a.geo.rec32 + td.rb, o);
    off[L::Q] = o;
    bytes = nrec > 0 ? (((uint32_t)((o + nrec) * (int)sizeof(uint32_t)) + 15u) & ~15u) : 0u;
    dst = stage + SL::kRec;
  }
  const uint32_t total = __reduce_add_sync(0xffffffffu, bytes + (src2 ? 16u : 0u));
  __syncwarp();
  if (lane == 0) mbar_arrive_expect_tx(bar, total);
  __syncwarp();
  if (bytes) bulk_copy_g2s(dst, src, bytes, bar);
  if (src2) bulk_copy_g2s(dst2, src2, 16u, bar);
}

// A link's coefficients through the read-only (non-coherent) path.  They do not
// change during a sweep, so the compiler may issue these loads ahead of the
// boundary block's stores (which it could not do with plain loads, since a store
// of the storage type may alias them); each load then costs one L2 round trip per
// warp instead of one per cut direction in turn.
template <class C>
__device__ __forceinline__ LinkCoef<C> load_coef_nc(const LinkCoef<C> *p) {
  LinkCoef<C> c;
  if constexpr (sizeof(C) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    c.a = v.x; c.bb = v.y; c.c = v.z; c.w = v.w;
  } else {
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    c.a = v0.x; c.bb = v0.y; c.c = v1.x; c.w = v1.y;
  }
  return c;
}

// Resident blocks per SM the register budget is sized for (launch bounds).  With
// 4- and 2-byte storage a block of a single-context sweep takes 44.5 KB (D3Q19),
// 35.8 KB (D3Q15) or 22.5 KB (D2Q9) of shared memory, so 5, 6 or 9 fit an SM: the
// register budget follows (96, 80 and 64 registers a thread, 5, 6 and 8 blocks).
// Batch sweeps read their members' arguments from memory into registers: D2Q9 keeps
// 96 registers (below that it spills, which costs more than the occupancy gains), the
// 3D lattices take 128 (4 blocks): with 96 they spill 40-200 bytes a thread, and a
// D3Q19 batch of tilted pipes runs 9 % faster at 4 blocks without spills than at 5
// with them.
#ifndef LBM_MINBLOCKS_F32
#define LBM_MINBLOCKS_F32 5
#endif
#ifndef LBM_MINBLOCKS_D2Q9
#define LBM_MINBLOCKS_D2Q9 8
#endif
#ifndef LBM_MINBLOCKS_D3Q15
#define LBM_MINBLOCKS_D3Q15 6
#endif
#ifndef LBM_MINBLOCKS_D3Q19_2B
#define LBM_MINBLOCKS_D3Q19_2B 5
#endif
#ifndef LBM_MINBLOCKS_BATCH_3D
#define LBM_MINBLOCKS_BATCH_3D 4
#endif
template <class L, class T, bool BATCH>
struct MinBlocks {
  static constexpr int value =
      BATCH ? (L::Q == 9 ? LBM_MINBLOCKS_F32 : LBM_MINBLOCKS_BATCH_3D)
            : (L::Q == 9 ? LBM_MINBLOCKS_D2Q9
                         : (L::Q == 15 ? LBM_MINBLOCKS_D3Q15
                                       : (sizeof(T) == 2 ? LBM_MINBLOCKS_D3Q19_2B : LBM_MINBLOCKS_F32)));
};
#ifndef LBM_MINBLOCKS_BATCH_F64
#define LBM_MINBLOCKS_BATCH_F64 2
#endif
template <class L, bool BATCH>
struct MinBlocks<L, double, BATCH> {
  // 4 x 128 threads: 128 registers (FP64 arithmetic).  Batches: 2 (the members'
  // arguments on top of the FP64 state spill 60-180 bytes a thread at 128 or 168
  // registers; 64-node FP64 tiles fit only 2 blocks' shared memory anyway)
  static constexpr int value = BATCH ? LBM_MINBLOCKS_BATCH_F64 : 4;
};

// One fused time step.  Persistent warps: global warp w handles tiles
// w, w + W_total, ...  I is the index type of a population slot (int when
// Q*S < 2^31, else long long).
// Shared-memory offset of a window's first element when every row starts on a
// 16-byte boundary (nx*sizeof(T) % 16 == 0): the copy of an odd-step window that
// begins at x0 - ex starts 16/sizeof(T) - 1 elements early for ex = +1, one element
// early for ex = -1, exactly for ex = 0.
template <class T>
__device__ __forceinline__ constexpr int aligned_window_offset(int ex) {
  return ex > 0 ? 16 / (int)sizeof(T) - 1 : (ex < 0 ? 1 : 0);
}

// Arguments of the instance a tile belongs to: the kernel parameter for a single
// context, an entry of the instance table for a batch.
template <bool BATCH, class C>
__device__ __forceinline__ const SweepArgs<C> &args_for(const SweepArgs<C> &a, const SweepArgs<C> *inst,
                                                       const int *tile_inst, int tile) {
  if constexpr (BATCH) return inst[tile_inst[tile]];
  else return a;
}

template <class L, class T, bool ODD, bool SKEW, bool ALIGNED, class I, bool BATCH, int TW = kTileW>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, MinBlocks<L, T, BATCH>::value)
    sweep_kernel(const SweepArgs<typename Storage<T>::C> a, const TileDesc *__restrict__ tiles,
                 int n_tiles, const SweepArgs<typename Storage<T>::C> *__restrict__ inst,
                 const int *__restrict__ tile_inst) {
  using C = typename Storage<T>::C;
  using SL = StageLayout<L, T, TW>;
  static_assert(SL::kRec % 16 == 0 && SL::kStage % 16 == 0, "bulk-copy destinations are 16-byte aligned");
  static_assert((StageShape<T, TW>::kWidth * sizeof(T)) % 16 == 0, "window stride");
  constexpr int Q = L::Q;
  constexpr int NS = StageShape<T, TW>::kStages;
  constexpr int W = StageShape<T, TW>::kWidth;
  constexpr int NO = SL::kNOff;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *wsm = smem_raw + (size_t)warp * warp_smem_bytes<L, T, TW>();
  uint64_t *bars = reinterpret_cast<uint64_t *>(wsm + SL::kBars);
  int *offs = reinterpret_cast<int *>(wsm + SL::kOffs);

  const int gw = blockIdx.x * kWarpsPerBlock + warp;
  const int nw = gridDim.x * kWarpsPerBlock;
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  for (int s = 0; s < NS; ++s) {
    const int tile = gw + s * nw;
    if (tile < n_tiles)
      issue_tile<L, T, ODD, ALIGNED, I, TW>(args_for<BATCH>(a, inst, tile_inst, tile), tiles[tile],
                               wsm + s * SL::kStage, offs + s * NO, &bars[s]);
  }

  int k = 0;
  for (int tile = gw; tile < n_tiles; tile += nw, ++k) {
    const int s = k % NS;
    // the detection wait is limited by the host-set a.wait_polls (lbm_set_wait_limit)
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)(k / NS) & 1u, a.wait_polls);
    if (__any_sync(0xffffffffu, !ok)) {
      // a copy did not land in time: flag it, then wait (with the long default
      // limit) for every copy this warp still has in flight into its shared
      // memory before leaving, and stop
      if (lane == 0) atomicOr(args_for<BATCH>(a, inst, tile_inst, tile).status, 2);
      for (int j = 0; j < NS; ++j)
        if (tile + j * nw < n_tiles) mbar_wait_bounded(&bars[(k + j) % NS], (uint32_t)((k + j) / NS) & 1u);
      return;
    }
    const SweepArgs<C> &A = args_for<BATCH>(a, inst, tile_inst, tile);
    T *__restrict__ pop = static_cast<T *>(A.pop);
    const I S = (I)A.S;
    const int nxm1 = A.nx - 1;
    const LinkCoef<C> *coef = static_cast<const LinkCoef<C> *>(A.geo.coef);
    T *const lnk = static_cast<T *>(A.geo.lnk);
    const TileDesc td = tiles[tile];
    const int y = td.yz & 0xffff, z = td.yz >> 16;
    const unsigned char *stg = wsm + s * SL::kStage;
    const T *st = reinterpret_cast<const T *>(stg);
    const uint32_t *rec_s = reinterpret_cast<const uint32_t *>(stg + SL::kRec) + offs[s * NO + Q];
    const int row = A.nx * (y + A.ny * z);
#pragma unroll 1
    for (int j = 0; j < TW / 32; ++j) {
    const int xl = j * 32 + lane;          // position inside the tile
    const int x = td.x0 + xl;
    const int n = row + x;
    const bool solid = (td.solid >> xl) & 1ull;
    int boff = 0;
    uint32_t bmask = 0u;
    if ((td.bnd >> xl) & 1ull) {
      const uint32_t r = rec_s[__popcll(td.bnd & ((1ull << xl) - 1ull))];
      bmask = r & ((1u << kRecShift) - 1u);
      boff = td.lb + (int)(r >> kRecShift);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(coef + boff));
    }
    C g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int o = ALIGNED ? (ODD ? aligned_window_offset<T>(L::ex(i)) : 0) : offs[s * NO + i];
      g[i] = Storage<T>::load(st + i * W + o + xl);
    }
    if (j == TW / 32 - 1) {
      __syncwarp();   // stage s consumed: refill it with the tile NS rounds ahead
      const int nt = tile + NS * nw;
      if (nt < n_tiles)
        issue_tile<L, T, ODD, ALIGNED, I, TW>(args_for<BATCH>(a, inst, tile_inst, nt), tiles[nt],
                                 wsm + s * SL::kStage, offs + s * NO, &bars[s]);
    }
    if (solid) continue;

    // lanes on the periodic x-edges: the row windows cannot follow the wrap.  A step
    // across x = 0 lands in column nx-1 of the row shifted by (+sy, +sz), across
    // x = nx-1 in column 0 of the row shifted by (-sy, -sz).
    const bool xlo = ODD && x == 0, xhi = ODD && x == nxm1;
    // node index in the row (y + dy, z + dz) shifted across the wrap, column xc
    auto across = [&](int xc, int dy, int dz) -> I {
      const int yy = wrap1(y + dy, A.ny);
      const int zz = L::D == 3 ? wrap1(z + dz, A.nz) : 0;
      return (I)xc + (I)A.nx * ((I)yy + (I)A.ny * zz);
    };
    const int sy = SKEW ? A.sy : 0, sz = SKEW ? A.sz : 0;
    // (a node can be on both edges when nx = 1)
    if (ODD && !ALIGNED && xlo) {          // aligned rows: staged with the windows
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (L::ex(i) > 0)
          g[i] = Storage<T>::load(pop + (I)L::opp(i) * S + across(nxm1, sy - L::ey(i), sz - L::ez(i)));
    }
    if (ODD && !ALIGNED && xhi) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        if (L::ex(i) < 0)
          g[i] = Storage<T>::load(pop + (I)L::opp(i) * S + across(0, -sy - L::ey(i), -sz - L::ez(i)));
    }
    if (ODD && bmask) {
      // populations that arrive through a cut link were left in the link buffer
      // by the previous (even) step
#pragma unroll
      for (int dd = 1; dd < Q; ++dd)
        if (bmask & (1u << dd))
            g[L::opp(dd)] = Storage<T>::load(lnk + boff + __popc(bmask & ((1u << dd) - 1u)));
    }

    if (A.save) {
#pragma unroll
      for (int i = 0; i < Q; ++i) A.save[(long long)i * A.N + n] = g[i];
    }

    C gp[Q];
    C drho;
    collide<L, C, T>(g, gp, A, drho);
    if (!(fabs(drho) < C(1e6))) atomicOr(A.status, 1);

    T *const pn = pop + n;
    if (!ODD) {
#pragma unroll
      for (int i = 0; i < Q; ++i) Storage<T>::store(pn + (I)A.koff_even[i], gp[i]);   // slot opp(i) of x
    } else {
      // rows y +- 1, z +- 1 stay inside the grid for the whole tile: constant offsets
      const bool rows_inside =
          y > 0 && y < A.ny - 1 && (L::D == 2 || (z > 0 && z < A.nz - 1));
      if (rows_inside) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const int ex = L::ex(i);
          if ((ex > 0 && xhi) || (ex < 0 && xlo)) continue;   // crosses the x-wrap
          Storage<T>::store(pn + (I)A.koff_odd[i], gp[i]);     // slot i of x + e_i
        }
        // stores across the periodic x-wrap: when the skew-shifted rows (y +- sy +
        // e_y, z +- sz + e_z) stay inside the grid, the target is the regular odd-step
        // offset moved by +-kwrap; otherwise every row index is wrapped
        if (xlo) {
          const int ys = y + sy, zs = z + sz;
          if (ys >= 1 && ys <= A.ny - 2 && (L::D == 2 || (zs >= 1 && zs <= A.nz - 2))) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
              if (L::ex(i) < 0) Storage<T>::store(pn + (I)(A.koff_odd[i] + A.kwrap), gp[i]);
          } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
              if (L::ex(i) < 0)
                Storage<T>::store(pop + (I)i * S + across(nxm1, sy + L::ey(i), sz + L::ez(i)), gp[i]);
          }
        }
        if (xhi) {
          const int ys = y - sy, zs = z - sz;
          if (ys >= 1 && ys <= A.ny - 2 && (L::D == 2 || (zs >= 1 && zs <= A.nz - 2))) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
              if (L::ex(i) > 0) Storage<T>::store(pn + (I)(A.koff_odd[i] - A.kwrap), gp[i]);
          } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
              if (L::ex(i) > 0)
                Storage<T>::store(pop + (I)i * S + across(0, -sy + L::ey(i), -sz + L::ez(i)), gp[i]);
          }
        }
      } else {
        // rows of the tile touch a periodic edge in y or z: wrap every neighbour
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const long long dn = wrap_index(x, y, z, L::ex(i), L::ey(i), L::ez(i), A.nx, A.ny, A.nz,
                                          A.sy, A.sz);
          Storage<T>::store(pop + (I)i * S + (I)dn, gp[i]);
        }
      }
    }

    // single-node boundary scheme on the cut links of this node (Eqs. 2.10, 2.13)
    if (bmask) {
#pragma unroll
      for (int dd = 1; dd < Q; ++dd) {
        if (bmask & (1u << dd)) {
          const int kk = boff + __popc(bmask & ((1u << dd) - 1u));
          const LinkCoef<C> c = load_coef_nc(coef + kk);
          const int i = L::opp(dd);
          const C v = A.one_minus_b * g[i] + c.a * g[dd] + c.bb * gp[i] + c.c * gp[dd] + c.w * A.wfac;
          if (!ODD) Storage<T>::store(lnk + kk, v);          // read by the next odd step
          else Storage<T>::store(pn + (I)i * S, v);          // slot i of x_f itself
        }
      }
    }
    }
  }
}

// Persistent grid size of one kernel instantiation on the current device
// (resident blocks per SM x SMs).  The first call on each device also raises the
// kernel's dynamic shared-memory limit there (a per-device function attribute) to
// what it uses; both are cached per device ordinal.
constexpr int kMaxDevices = 64;
template <auto Kernel>
int persistent_blocks(int threads, size_t smem) {
  static std::mutex mu;
  static int cached[kMaxDevices] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (cached[dev] == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, threads, smem);
    cached[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  return cached[dev];
}

template <auto Kernel, class A>
void launch_persistent(const A &a, const TileDesc *tiles, int n_tiles, size_t smem, cudaStream_t st,
                       const A *inst = nullptr, const int *tile_inst = nullptr, int blocks_per_sm = 0,
                       bool prepare_only = false) {
  const int threads = kWarpsPerBlock * 32;
  int grid = persistent_blocks<Kernel>(threads, smem);
  if (blocks_per_sm > 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks_per_sm * sms < grid) grid = blocks_per_sm * sms;
  }
  const int need = (n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (grid > need) grid = need;
  if (!prepare_only) Kernel<<<grid, threads, smem, st>>>(a, tiles, n_tiles, inst, tile_inst);
}

// Tile width of the single-context sweep per storage type: 64 nodes, or 32-node
// half tiles for FP64 storage (see StageShape; on the L = 256 pipe 3.99 instead of
// 4.01 ms per step, the same with 64-node tiles in one stage or 32-node tiles in 3).
#ifndef LBM_TILEW_F64
#define LBM_TILEW_F64 32
#endif
#ifndef LBM_TILEW_4B
#define LBM_TILEW_4B 64
#endif
#ifndef LBM_TILEW_2B
#define LBM_TILEW_2B 64
#endif
template <class T>
constexpr int single_tile_w() {
  return sizeof(T) == 8 ? LBM_TILEW_F64 : (sizeof(T) == 4 ? LBM_TILEW_4B : LBM_TILEW_2B);
}

template <class L, class T>
cudaError_t launch_sweep_t(bool odd, const SweepArgs<typename Storage<T>::C> &a, const TileDesc *tiles64,
                           int n_tiles64, const TileDesc *tiles_half, int n_half, cudaStream_t st) {
  constexpr int TW = single_tile_w<T>();
  const TileDesc *tiles = TW == kTileW ? tiles64 : tiles_half;
  const int n_tiles = TW == kTileW ? n_tiles64 : n_half;
  if (n_tiles == 0) return cudaSuccess;
  const bool skew = a.sy != 0 || a.sz != 0;
  const bool big = (long long)L::Q * a.S >= (1LL << 31);
  const size_t smem = kWarpsPerBlock * warp_smem_bytes<L, T, TW>();
  const bool aligned = ((long long)a.nx * (long long)sizeof(T)) % 16 == 0;
#define LBM_LAUNCH(O, S, I)                                                                              \
  do {                                                                                                   \
    if (aligned) launch_persistent<sweep_kernel<L, T, O, S, true, I, false, TW>>(a, tiles, n_tiles, smem, st);  \
    else launch_persistent<sweep_kernel<L, T, O, S, false, I, false, TW>>(a, tiles, n_tiles, smem, st);        \
  } while (0)
  if (big) {
    if (odd) { if (skew) LBM_LAUNCH(true, true, long long); else LBM_LAUNCH(true, false, long long); }
    else LBM_LAUNCH(false, false, long long);
  } else {
    if (odd) { if (skew) LBM_LAUNCH(true, true, int); else LBM_LAUNCH(true, false, int); }
    else LBM_LAUNCH(false, false, int);
  }
#undef LBM_LAUNCH
  return cudaGetLastError();
}

// One step of a batch: the tiles of one kernel class of members in one persistent
// launch, each tile reading its member's arguments from the table.  aligned: every
// member's rows start on 16-byte boundaries (aligned-window path); skew: some
// member has a skewed x-wrap.  Batches whose slots need 64-bit indices (big) use
// the general kernel (unaligned windows, skew) for every member, in 64-node tiles.
// TW: the width of the tiles in the list (64, or 32 for lists of half tiles).
// prepare_only: set up the kernel's launch attributes without launching (done once
// before a stream capture).
template <class L, class T, int TW>
cudaError_t launch_sweep_batch_t(bool odd, const SweepArgs<typename Storage<T>::C> *inst,
                                 const TileDesc *tiles, const int *tile_inst, int n_tiles,
                                 bool big, bool aligned, bool skew, int blocks_per_sm, cudaStream_t st,
                                 bool prepare_only) {
  if (n_tiles == 0) return cudaSuccess;
  using A = SweepArgs<typename Storage<T>::C>;
  const size_t smem = kWarpsPerBlock * warp_smem_bytes<L, T, TW>();
  A dummy{};
  dummy.wait_polls = kWaitLimit;
#define LBM_LAUNCH_B(O, S, AL, I)                                                                      \
  launch_persistent<sweep_kernel<L, T, O, S, AL, I, true, TW>>(dummy, tiles, n_tiles, smem, st, inst,  \
                                                               tile_inst, blocks_per_sm, prepare_only)
  if (big) {
    if constexpr (TW != kTileW) {
      return cudaErrorInvalidValue;   // 64-bit slot indices: 64-node tiles only
    } else {
      if (odd) LBM_LAUNCH_B(true, true, false, long long);
      else LBM_LAUNCH_B(false, false, false, long long);
    }
  } else if (!odd) {
    if (aligned) LBM_LAUNCH_B(false, false, true, int);
    else LBM_LAUNCH_B(false, false, false, int);
  } else if (aligned) {
    if (skew) LBM_LAUNCH_B(true, true, true, int);
    else LBM_LAUNCH_B(true, false, true, int);
  } else {
    if (skew) LBM_LAUNCH_B(true, true, false, int);
    else LBM_LAUNCH_B(true, false, false, int);
  }
#undef LBM_LAUNCH_B
  return cudaGetLastError();
}

}  // namespace lbm
