// lattice.h -- compile-time lattice tables shared by the host and device code of
// the library (never by the oracle).
//
// D2Q9: velocities, weights and the transformation matrix M of the paper's
//   Appendix.  M is written as the Lallemand-Luo polynomial moments
//   1, 3|e|^2-4, (9|e|^4-21|e|^2+8)/2, e_x, (3|e|^2-5)e_x, e_y, (3|e|^2-5)e_y,
//   e_x^2-e_y^2, e_x e_y, which evaluate on the Appendix velocities to the printed
//   integer table.
// D3Q19: the 3D MRT model of d'Humieres et al. (2002), which the Appendix cites;
//   moments 1, 19|e|^2-30, (21|e|^4-53|e|^2+24)/2, e_x, (5|e|^2-9)e_x, e_y, ...,
//   3e_x^2-|e|^2, (3|e|^2-5)(3e_x^2-|e|^2), e_y^2-e_z^2, (3|e|^2-5)(e_y^2-e_z^2),
//   e_x e_y, e_y e_z, e_x e_z, (e_y^2-e_z^2)e_x, (e_z^2-e_x^2)e_y, (e_x^2-e_y^2)e_z.
//
// Every table is a constexpr function so that, inside fully unrolled loops, each
// entry is a literal and multiplications by 0 and +-1 fold away.
#pragma once

#ifdef __CUDACC__
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

namespace lbm {

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  static constexpr int kLattice = 0;
  LBM_HD static constexpr int ex(int i) {
    constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    return t[i];
  }
  LBM_HD static constexpr int ey(int i) {
    constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return t[i];
  }
  LBM_HD static constexpr int ez(int) { return 0; }
  LBM_HD static constexpr int opp(int i) {
    constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    return t[i];
  }
  // opp for a runtime index (no table): 1..4 and 5..8 are cycles of four
  LBM_HD static constexpr int opp_rt(int i) {
    return i == 0 ? 0 : (i < 5 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
  }
  // weight w_i times 36
  LBM_HD static constexpr int w36(int i) { return i == 0 ? 16 : (i < 5 ? 4 : 1); }
  LBM_HD static constexpr double w(int i) { return w36(i) / 36.0; }
  LBM_HD static constexpr int M(int k, int i) {
    const int x = ex(i), y = ey(i), r2 = x * x + y * y;
    switch (k) {
      case 0: return 1;
      case 1: return 3 * r2 - 4;
      case 2: return (9 * r2 * r2 - 21 * r2 + 8) / 2;
      case 3: return x;
      case 4: return (3 * r2 - 5) * x;
      case 5: return y;
      case 6: return (3 * r2 - 5) * y;
      case 7: return x * x - y * y;
      default: return x * y;
    }
  }
  LBM_HD static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5; }
  // pairs (i, opp(i)) with i the first member
  static constexpr int NP = 4;
  LBM_HD static constexpr int pair_first(int p) {
    constexpr int t[4] = {1, 2, 5, 6};
    return t[p];
  }
  // sum_i e_ix^2 = squared norm of the j rows
  static constexpr int kNormJ = 6;
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  static constexpr int kLattice = 1;
  LBM_HD static constexpr int ex(int i) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
  }
  LBM_HD static constexpr int ey(int i) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[i];
  }
  LBM_HD static constexpr int ez(int i) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[i];
  }
  LBM_HD static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
  LBM_HD static constexpr int opp_rt(int i) { return opp(i); }
  LBM_HD static constexpr int w36(int i) {
    return i == 0 ? 12 : (i < 7 ? 2 : 1);
  }
  LBM_HD static constexpr double w(int i) { return w36(i) / 36.0; }
  LBM_HD static constexpr int M(int k, int i) {
    const int x = ex(i), y = ey(i), z = ez(i), r2 = x * x + y * y + z * z;
    switch (k) {
      case 0: return 1;
      case 1: return 19 * r2 - 30;
      case 2: return (21 * r2 * r2 - 53 * r2 + 24) / 2;
      case 3: return x;
      case 4: return (5 * r2 - 9) * x;
      case 5: return y;
      case 6: return (5 * r2 - 9) * y;
      case 7: return z;
      case 8: return (5 * r2 - 9) * z;
      case 9: return 3 * x * x - r2;
      case 10: return (3 * r2 - 5) * (3 * x * x - r2);
      case 11: return y * y - z * z;
      case 12: return (3 * r2 - 5) * (y * y - z * z);
      case 13: return x * y;
      case 14: return y * z;
      case 15: return x * z;
      case 16: return (y * y - z * z) * x;
      case 17: return (z * z - x * x) * y;
      default: return (x * x - y * y) * z;
    }
  }
  LBM_HD static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5 || k == 7; }
  static constexpr int NP = 9;
  LBM_HD static constexpr int pair_first(int p) { return 2 * p + 1; }
  static constexpr int kNormJ = 10;
};

// D3Q15 of the paper's Appendix: velocities in the printed order (rest; +x,-x,+y,-y,
// +z,-z; then the eight corners (1,1,1), (-1,1,1), (1,-1,1), (-1,-1,1), (1,1,-1),
// (-1,1,-1), (1,-1,-1), (-1,-1,-1)), weights 2/9, 1/9, 1/72, and the printed M,
// whose rows are the polynomials 1, |e|^2-2, (15|e|^4-55|e|^2+32)/2, e_x,
// (5|e|^2-13)e_x/2, e_y, (5|e|^2-13)e_y/2, e_z, (5|e|^2-13)e_z/2, 3e_x^2-|e|^2,
// e_y^2-e_z^2, e_x e_y, e_y e_z, e_x e_z, e_x e_y e_z.
struct D3Q15 {
  static constexpr int Q = 15;
  static constexpr int D = 3;
  static constexpr int kLattice = 2;
  LBM_HD static constexpr int ex(int i) {
    constexpr int t[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[i];
  }
  LBM_HD static constexpr int ey(int i) {
    constexpr int t[15] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
  }
  LBM_HD static constexpr int ez(int i) {
    constexpr int t[15] = {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return t[i];
  }
  // faces pair as (1,2), (3,4), (5,6); corner i pairs with 21 - i
  LBM_HD static constexpr int opp(int i) {
    return i == 0 ? 0 : (i < 7 ? ((i & 1) ? i + 1 : i - 1) : 21 - i);
  }
  LBM_HD static constexpr int opp_rt(int i) { return opp(i); }
  LBM_HD static constexpr double w(int i) { return i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0); }
  LBM_HD static constexpr int M(int k, int i) {
    const int x = ex(i), y = ey(i), z = ez(i), r2 = x * x + y * y + z * z;
    switch (k) {
      case 0: return 1;
      case 1: return r2 - 2;
      case 2: return (15 * r2 * r2 - 55 * r2 + 32) / 2;
      case 3: return x;
      case 4: return (5 * r2 - 13) * x / 2;
      case 5: return y;
      case 6: return (5 * r2 - 13) * y / 2;
      case 7: return z;
      case 8: return (5 * r2 - 13) * z / 2;
      case 9: return 3 * x * x - r2;
      case 10: return y * y - z * z;
      case 11: return x * y;
      case 12: return y * z;
      case 13: return x * z;
      default: return x * y * z;
    }
  }
  LBM_HD static constexpr bool conserved(int k) { return k == 0 || k == 3 || k == 5 || k == 7; }
  static constexpr int NP = 7;
  LBM_HD static constexpr int pair_first(int p) {
    constexpr int t[7] = {1, 3, 5, 7, 8, 9, 10};
    return t[p];
  }
  static constexpr int kNormJ = 10;
};

// Runtime (non-constant index) access to the velocity components and opposites,
// from bit masks built at compile time, so that no table lands in local memory.
template <class L>
constexpr unsigned comp_mask(int comp, int sign) {
  unsigned m = 0;
  for (int i = 0; i < L::Q; ++i) {
    const int v = comp == 0 ? L::ex(i) : (comp == 1 ? L::ey(i) : L::ez(i));
    if (v == sign) m |= 1u << i;
  }
  return m;
}
template <class L>
struct DirBits {
  static constexpr unsigned kXp = comp_mask<L>(0, 1), kXn = comp_mask<L>(0, -1);
  static constexpr unsigned kYp = comp_mask<L>(1, 1), kYn = comp_mask<L>(1, -1);
  static constexpr unsigned kZp = comp_mask<L>(2, 1), kZn = comp_mask<L>(2, -1);
  LBM_HD static int ex(int i) { return (int)((kXp >> i) & 1u) - (int)((kXn >> i) & 1u); }
  LBM_HD static int ey(int i) { return (int)((kYp >> i) & 1u) - (int)((kYn >> i) & 1u); }
  LBM_HD static int ez(int i) { return (int)((kZp >> i) & 1u) - (int)((kZn >> i) & 1u); }
};

// squared norm of row k: sum_i M(k,i)^2
template <class L>
LBM_HD constexpr int row_norm2(int k) {
  int s = 0;
  for (int i = 0; i < L::Q; ++i) s += L::M(k, i) * L::M(k, i);
  return s;
}

// parity of row k under e -> -e: odd rows satisfy M(k, opp(i)) = -M(k, i),
// even rows M(k, opp(i)) = M(k, i)
template <class L>
LBM_HD constexpr bool row_is_odd(int k) {
  if (L::M(k, 0) != 0) return false;
  for (int p = 0; p < L::NP; ++p) {
    const int i = L::pair_first(p);
    if (L::M(k, i) != -L::M(k, L::opp(i))) return false;
  }
  return true;
}
template <class L>
LBM_HD constexpr bool row_is_even(int k) {
  for (int p = 0; p < L::NP; ++p) {
    const int i = L::pair_first(p);
    if (L::M(k, i) != L::M(k, L::opp(i))) return false;
  }
  return true;
}
template <class L>
constexpr bool lattice_is_consistent() {
  for (int i = 0; i < L::Q; ++i)
    if (L::opp_rt(i) != L::opp(i)) return false;
  // every row has a parity, rows are orthogonal, pairs cover every moving direction
  for (int k = 0; k < L::Q; ++k)
    if (row_is_odd<L>(k) == row_is_even<L>(k)) return false;
  for (int a = 0; a < L::Q; ++a)
    for (int b = 0; b < L::Q; ++b) {
      if (a == b) continue;
      int s = 0;
      for (int i = 0; i < L::Q; ++i) s += L::M(a, i) * L::M(b, i);
      if (s != 0) return false;
    }
  int seen = 0;
  for (int p = 0; p < L::NP; ++p) {
    const int i = L::pair_first(p);
    if (L::opp(i) == i || L::ex(i) != -L::ex(L::opp(i)) || L::ey(i) != -L::ey(L::opp(i)) ||
        L::ez(i) != -L::ez(L::opp(i)))
      return false;
    seen += 2;
  }
  return seen == L::Q - 1;
}
static_assert(lattice_is_consistent<D2Q9>(), "D2Q9 tables");
static_assert(lattice_is_consistent<D3Q19>(), "D3Q19 tables");
static_assert(row_norm2<D2Q9>(1) == 36 && row_norm2<D2Q9>(3) == D2Q9::kNormJ, "D2Q9 norms");
static_assert(row_norm2<D3Q19>(1) == 2394 && row_norm2<D3Q19>(3) == D3Q19::kNormJ, "D3Q19 norms");
static_assert(lattice_is_consistent<D3Q15>(), "D3Q15 tables");
static_assert(row_norm2<D3Q15>(1) == 18 && row_norm2<D3Q15>(2) == 360 && row_norm2<D3Q15>(3) == D3Q15::kNormJ &&
                  row_norm2<D3Q15>(4) == 40 && row_norm2<D3Q15>(14) == 8,
              "D3Q15 norms");
// the printed table's entries
static_assert(D3Q15::M(2, 0) == 16 && D3Q15::M(2, 1) == -4 && D3Q15::M(2, 7) == 1 &&
                  D3Q15::M(4, 1) == -4 && D3Q15::M(4, 2) == 4 && D3Q15::M(4, 7) == 1 &&
                  D3Q15::M(11, 8) == -1 && D3Q15::M(14, 12) == 1 && D3Q15::M(14, 14) == -1,
              "D3Q15 M");

}  // namespace lbm
