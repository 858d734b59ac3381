// lbm_capi.cu -- the C-ABI of include/lbm.h: context, argument validation,
// geometry compaction (cut links of Sec. 2 into per-node records and per-link
// coefficients of Eq. 2.13), and the host side of every call.  All arithmetic of
// a time step runs in the kernels (sweep_*.cu, aux_kernels.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lbm.h"
#include "lattice.h"
#include "lbm_internal.h"

namespace lbm {
cudaError_t launch_sweep_d2q9(int, bool, const SweepArgs<double> &, const SweepArgs<float> &,
                               const TileDesc *, int, const TileDesc *, int, cudaStream_t);
cudaError_t launch_sweep_d3q19(int, bool, const SweepArgs<double> &, const SweepArgs<float> &,
                               const TileDesc *, int, const TileDesc *, int, cudaStream_t);
cudaError_t launch_sweep_d3q15(int, bool, const SweepArgs<double> &, const SweepArgs<float> &,
                               const TileDesc *, int, const TileDesc *, int, cudaStream_t);
int error_norms_noalloc(int device, int lattice, int precision, const AuxArgs &a, bool odd,
                        const double *u_ref, double *out, cudaStream_t st, const char **why);
cudaError_t launch_sweep_batch_d2q9(int, int, bool, const void *, const TileDesc *, const int *,
                                   int, bool, bool, bool, int, cudaStream_t, bool);
cudaError_t launch_sweep_batch_d3q19(int, int, bool, const void *, const TileDesc *, const int *,
                                   int, bool, bool, bool, int, cudaStream_t, bool);
cudaError_t launch_sweep_batch_d3q15(int, int, bool, const void *, const TileDesc *, const int *,
                                   int, bool, bool, bool, int, cudaStream_t, bool);
cudaError_t launch_sweep(int lattice, int precision, bool odd, const SweepArgs<double> &a64,
                         const SweepArgs<float> &a32, const TileDesc *tiles, int n_tiles,
                         const TileDesc *tiles_half, int n_half, cudaStream_t st) {
  switch (lattice) {
    case LBM_D2Q9: return launch_sweep_d2q9(precision, odd, a64, a32, tiles, n_tiles, tiles_half, n_half, st);
    case LBM_D3Q15: return launch_sweep_d3q15(precision, odd, a64, a32, tiles, n_tiles, tiles_half, n_half, st);
    default: return launch_sweep_d3q19(precision, odd, a64, a32, tiles, n_tiles, tiles_half, n_half, st);
  }
}
}  // namespace lbm

using namespace lbm;

// What a forward pass of the adjoint leaves for the backward pass: its start time,
// length, checkpoint interval and checkpoint times, and the identity of the state
// it ended in (state serial and argument version), which the backward pass checks.
struct AdjTape {
  bool valid = false;
  bool last_saved = false;      // the last segment's states are still in the workspace
  long long t0 = 0, T = 0, K = 0, nseg = 0;
  std::vector<long long> tck;
  long long serial = -1, version = -1;
};

struct lbm_ctx {
  int lattice = 0, Q = 0, D = 0, precision = 0;
  int nx = 0, ny = 0, nz = 0, sy = 0, sz = 0;
  long long N = 0;
  double rho0 = 1.0;
  double s[19] = {0};
  double c0 = 0.0, c1 = 1.0, c2 = 0.0, b = 1.0;
  bool allow_nonconvex = false;
  double g[3] = {0, 0, 0};
  int device = 0;
  cudaStream_t stream = nullptr;
  long long t = 0;
  int wait_polls = kWaitLimitDefault;  // lbm_set_wait_limit
  double wf_a0 = 1.0, wf_r = 1.0;  // wall-velocity factor a0 r^(t - wf_t0)
  long long wf_t0 = 0;
  bool geometry_set = false;
  bool two_node = false;        // Eq. 2.11 on links whose x_l is fluid
  TwoNodeLink *tn = nullptr;
  long long n_tn = 0;
  void *tn_delta = nullptr;

  // device buffers
  void *pop_alloc = nullptr;    // populations with kPopPadBytes on both sides
  void *pop = nullptr;          // = pop_alloc + kPopPadBytes
  uint8_t *cls = nullptr;
  int32_t *bidx = nullptr;
  uint32_t *bmask = nullptr;
  int32_t *boff = nullptr;
  uint32_t *rec32 = nullptr;    // packed records of boundary nodes
  void *coef = nullptr;
  void *lnk = nullptr;          // boundary values carried from an even to an odd step
  int *status = nullptr;
  double *partials = nullptr;   // norm reduction scratch
  double *norm_out = nullptr;
  double *u_ref = nullptr;
  double *u_prev = nullptr;
  double *mom_rho = nullptr;
  double *mom_u = nullptr;
  TileDesc *tiles = nullptr;    // active 64-node tiles of the sweep
  int n_tiles = 0;
  TileDesc *tiles_half = nullptr;  // the same tiles cut into 32-node halves
  int n_tiles_half = 0;

  // host copy of the cut links in device order (for re-deriving coefficients)
  std::vector<int32_t> link_dir;
  std::vector<int64_t> link_node;
  std::vector<double> link_q;
  std::vector<double> link_uw;  // 3 per link
  std::vector<int64_t> link_src; // input position of the link at each device position
  // device workspace of lbm_adjoint (pointer, capacity), kept between calls
  std::pair<void *, size_t> adj_ws[13] = {};
  AdjTape tape;                 // what lbm_adjoint_forward left for the backward pass
  long long state_serial = 0;   // bumped by every call that changes the populations
  long long n_links = 0, n_fluid = 0, n_boundary = 0;

  SweepArgs<double> a64;
  SweepArgs<float> a32;
  long long version = 0;        // bumped whenever the sweep arguments change
  std::string err;
};

static std::string g_create_error = "no error";

static int fail(lbm_ctx *c, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return code;
}

#define CUDA_OR_FAIL(ctx, call)                                                      \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,     \
                  "%s: %s", #call, cudaGetErrorString(e_));                          \
  } while (0)

static int store_bytes(int precision) {
  return precision == LBM_F64 ? 8 : (precision == LBM_F32_DEV ? 4 : 2);
}

// guard bytes after the node-class and record arrays (aligned window copies)
constexpr size_t kGuardBytes = 1024;

static size_t pop_alloc_bytes(const lbm_ctx *c) {
  return (size_t)c->Q * slot_stride(c->N) * store_bytes(c->precision) + 2 * kPopPadBytes;
}

// bytes of the link buffer: one storage element per cut link
static size_t link_bytes(const lbm_ctx *c) {
  return (size_t)store_bytes(c->precision) * std::max<long long>(1, c->n_links);
}

template <class F>
static auto with_lat(int lattice, F &&f) {
  return lattice == LBM_D2Q9 ? f(D2Q9{}) : (lattice == LBM_D3Q15 ? f(D3Q15{}) : f(D3Q19{}));
}

static long long wrap_host(const lbm_ctx *c, int x, int y, int z, int dx, int dy, int dz) {
  int xs = x + dx, ys = y + dy, zs = z + dz;
  if (xs < 0) { xs += c->nx; ys += c->sy; zs += c->sz; }
  else if (xs >= c->nx) { xs -= c->nx; ys -= c->sy; zs -= c->sz; }
  if (ys < 0) ys += c->ny; else if (ys >= c->ny) ys -= c->ny;
  if (zs < 0) zs += c->nz; else if (zs >= c->nz) zs -= c->nz;
  return xs + (long long)c->nx * (ys + (long long)c->ny * zs);
}

static AuxArgs aux_args(const lbm_ctx *c) {
  AuxArgs a;
  a.pop = c->pop;
  a.N = c->N;
  a.S = slot_stride(c->N);
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.sy = c->sy; a.sz = c->sz;
  a.cls = c->cls;
  a.bidx = c->bidx;
  a.bmask = c->bmask;
  a.boff = c->boff;
  a.lnk = c->lnk;
  a.rho0 = c->rho0;
  for (int k = 0; k < 3; ++k) a.g[k] = c->g[k];
  return a;
}

// wall-velocity factor a0 r^(t - t0) of step t (lbm_set_wall_factor)
static double wall_factor(const lbm_ctx *c, long long t) {
  return c->wf_a0 * std::pow(c->wf_r, (double)(t - c->wf_t0));
}
static void set_step_factor(lbm_ctx *c, long long t) {
  const double a = wall_factor(c, t);
  c->a64.wfac = a;
  c->a32.wfac = (float)a;
}

static void refresh_args(lbm_ctx *c) {
  DevGeometry geo;
  geo.cls = c->cls; geo.bidx = c->bidx; geo.bmask = c->bmask; geo.boff = c->boff;
  geo.rec32 = c->rec32;
  geo.coef = c->coef;
  geo.lnk = c->lnk;
  auto fill = [&](auto &a) {
    using C = std::remove_reference_t<decltype(a.inv_rho0)>;
    a.pop = c->pop;
    a.N = c->N;
    a.S = slot_stride(c->N);
    a.nx = c->nx; a.ny = c->ny; a.nz = c->nz; a.sy = c->sy; a.sz = c->sz;
    a.geo = geo;
    with_lat(c->lattice, [&](auto lat) {
      using L = decltype(lat);
      for (int k = 0; k < 19; ++k) a.sn[k] = C(0);
      for (int k = 0; k < L::Q; ++k)
        if (!L::conserved(k)) a.sn[k] = C(c->s[k] / row_norm2<L>(k));
      for (int k = 0; k < 3; ++k) a.F[k] = C(c->rho0 * c->g[k] / L::kNormJ);
      if (L::D == 2) a.F[2] = C(0);
      return 0;
    });
    a.inv_rho0 = C(1.0 / c->rho0);
    a.one_minus_b = C(1.0 - c->b);
    a.wfac = C(wall_factor(c, c->t));
    a.status = c->status;
    a.wait_polls = c->wait_polls;
    with_lat(c->lattice, [&](auto lat) {
      using L = decltype(lat);
      const long long S = slot_stride(c->N), nxl = c->nx, nxy = (long long)c->nx * c->ny;
      for (int i = 0; i < 19; ++i) a.koff_even[i] = a.koff_odd[i] = 0;
      for (int i = 0; i < L::Q; ++i) {
        a.koff_even[i] = L::opp(i) * S;
        a.koff_odd[i] = i * S + L::ex(i) + nxl * L::ey(i) + nxy * L::ez(i);
      }
      a.kwrap = nxl * (1 + c->sy) + nxy * c->sz;
      return 0;
    });
  };
  fill(c->a64);
  fill(c->a32);
  ++c->version;
}

// l(gamma) of the family (Sec. 2 / Sec. 3 rules)
static double l_of(const lbm_ctx *c, double q) { return c->c0 + c->c1 * q + c->c2 * q * q; }

// Eq. 2.12
static bool convex(double q, double l) {
  return l >= std::max(0.0, 2.0 * q - 1.0) && l <= 2.0 * q;
}

// coefficients of Eq. 2.13 (b folded in) for every link, uploaded in the
// compute type of the storage precision
static int upload_coefficients(lbm_ctx *c) {
  const long long nl = c->n_links;
  if (nl == 0) return LBM_OK;
  std::vector<double> co(4 * nl);
  with_lat(c->lattice, [&](auto lat) {
    using L = decltype(lat);
    for (long long k = 0; k < nl; ++k) {
      const int d = c->link_dir[k];
      const int i = L::opp(d);
      const double q = c->link_q[k];
      const double l = l_of(c, q);
      const double inv = 1.0 / (1.0 + l);
      const double A = (1.0 + l - 2.0 * q) * inv;       // on f_ib(x_f, t), ib = d
      const double B = l * inv;                         // on f'_i(x_f, t)
      const double Cc = (2.0 * q - l) * inv;            // on f'_ib(x_f, t)
      const double edotphi = L::ex(i) * c->link_uw[3 * k] + L::ey(i) * c->link_uw[3 * k + 1] +
                             L::ez(i) * c->link_uw[3 * k + 2];
      // 2/(1+l) w_i rho0 e_i.phi / c_s^2 with c_s^2 = 1/3
      const double W = 2.0 * inv * L::w(i) * c->rho0 * edotphi * 3.0;
      co[4 * k + 0] = c->b * A;
      co[4 * k + 1] = c->b * B;
      co[4 * k + 2] = c->b * Cc;
      co[4 * k + 3] = c->b * W;
    }
    return 0;
  });
  if (c->precision == LBM_F64) {
    CUDA_OR_FAIL(c, cudaMemcpy(c->coef, co.data(), sizeof(double) * co.size(),
                               cudaMemcpyHostToDevice));
  } else {
    std::vector<float> cf(co.begin(), co.end());
    CUDA_OR_FAIL(c, cudaMemcpy(c->coef, cf.data(), sizeof(float) * cf.size(),
                               cudaMemcpyHostToDevice));
  }
  return LBM_OK;
}

// buffer `slot` of the adjoint's workspace with at least `bytes`, grown when needed
static cudaError_t adj_ws_get(lbm_ctx *c, int slot, size_t bytes, void **p) {
  auto &e = c->adj_ws[slot];
  if (e.second < bytes) {
    cudaFree(e.first);
    e = {nullptr, 0};
    const cudaError_t r = cudaMalloc(&e.first, bytes);
    if (r != cudaSuccess) {
      e.first = nullptr;
      return r;
    }
    e.second = bytes;
  }
  *p = e.first;
  return cudaSuccess;
}
static void adj_ws_free(lbm_ctx *c) {
  c->tape.valid = false;
  for (auto &e : c->adj_ws) {
    cudaFree(e.first);
    e = {nullptr, 0};
  }
}

static void free_two_node(lbm_ctx *c) {
  cudaFree(c->tn); c->tn = nullptr;
  cudaFree(c->tn_delta); c->tn_delta = nullptr;
  c->n_tn = 0;
}

// device list of the links whose node behind the boundary node, x_l = x_f + e_i,
// is fluid (the others keep the single-node value)
static int build_two_node(lbm_ctx *c) {
  free_two_node(c);
  if (!c->two_node || c->n_links == 0) return LBM_OK;
  std::vector<uint8_t> cls(c->N);
  CUDA_OR_FAIL(c, cudaMemcpy(cls.data(), c->cls, c->N, cudaMemcpyDeviceToHost));
  std::vector<TwoNodeLink> h;
  with_lat(c->lattice, [&](auto lat) {
    using L = decltype(lat);
    for (long long k = 0; k < c->n_links; ++k) {
      const long long n = c->link_node[k];
      const int d = c->link_dir[k], i = L::opp(d);
      const int x = (int)(n % c->nx);
      const long long r = n / c->nx;
      const long long xl = wrap_host(c, x, (int)(r % c->ny), (int)(r / c->ny), L::ex(i), L::ey(i), L::ez(i));
      if (cls[xl] != kSolid) h.push_back(TwoNodeLink{n, xl, (int)k, d});
    }
    return 0;
  });
  c->n_tn = (long long)h.size();
  if (h.empty()) return LBM_OK;
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->tn, sizeof(TwoNodeLink) * h.size()));
  CUDA_OR_FAIL(c, cudaMemcpy(c->tn, h.data(), sizeof(TwoNodeLink) * h.size(), cudaMemcpyHostToDevice));
  CUDA_OR_FAIL(c, cudaMalloc(&c->tn_delta, (c->precision == LBM_F64 ? 8 : 4) * h.size()));
  return LBM_OK;
}


static void free_geometry(lbm_ctx *c) {
  free_two_node(c);
  cudaFree(c->bidx); c->bidx = nullptr;
  cudaFree(c->bmask); c->bmask = nullptr;
  cudaFree(c->boff); c->boff = nullptr;
  cudaFree(c->coef); c->coef = nullptr;
  cudaFree(c->lnk); c->lnk = nullptr;
}

// 64-node tiles cut into 32-node halves; halves without a fluid node are dropped.
// A half keeps the tile's link-buffer base (its records' offsets are relative to it);
// the second half's records start after the first half's.  Lanes past a half are
// marked solid.
static void half_tiles(const std::vector<TileDesc> &in, std::vector<TileDesc> &out) {
  constexpr uint64_t kLo = 0xffffffffull;
  out.clear();
  out.reserve(2 * in.size());
  for (const TileDesc &d : in) {
    TileDesc a = d, h = d;
    a.solid = d.solid | ~kLo;
    a.bnd = d.bnd & kLo;
    h.x0 = d.x0 + 32;
    h.rb = d.rb + __builtin_popcountll(d.bnd & kLo);
    h.solid = (d.solid >> 32) | ~kLo;
    h.bnd = d.bnd >> 32;
    if ((a.solid & kLo) != kLo) out.push_back(a);
    if ((h.solid & kLo) != kLo) out.push_back(h);
  }
}

// Tile descriptors (see TileDesc) of every run of kTileW nodes along x that holds
// at least one fluid node, and the packed records of the boundary nodes, in node
// order.  solid == nullptr: an all-fluid box without cut links.
static int upload_tiles(lbm_ctx *c, const uint8_t *solid, const std::vector<uint8_t> *cls,
                        const std::vector<uint32_t> *bmask, const std::vector<int32_t> *boff) {
  if (c->ny > 65535 || c->nz > 65535)
    return fail(c, LBM_EINVAL, "grid: ny and nz must be below 65536");
  const int nxb = (c->nx + kTileW - 1) / kTileW;
  std::vector<TileDesc> t;
  t.reserve((size_t)nxb * c->ny * c->nz);
  std::vector<uint32_t> rec32;
  if (bmask) rec32.reserve(bmask->size());
  int rb = 0;
  for (int z = 0; z < c->nz; ++z)
    for (int y = 0; y < c->ny; ++y)
      for (int xb = 0; xb < nxb; ++xb) {
        const int x0 = xb * kTileW;
        const long long row = (long long)c->nx * (y + (long long)c->ny * z);
        TileDesc d{};
        d.x0 = x0;
        d.yz = y | (z << 16);
        d.rb = rb;
        d.lb = 0;
        bool any = false;
        for (int k = 0; k < kTileW; ++k) {
          const int x = x0 + k;
          const bool is_solid = x >= c->nx || (solid && solid[row + x]);
          if (is_solid) { d.solid |= 1ull << k; continue; }
          any = true;
          if (cls && (*cls)[row + x] == kBoundary) {
            const uint32_t m = (*bmask)[rb], off = (uint32_t)(*boff)[rb];
            if (!d.bnd) d.lb = (int)off;
            d.bnd |= 1ull << k;
            rec32.push_back(m | ((off - (uint32_t)d.lb) << kRecShift));
            ++rb;
          }
        }
        if (any) t.push_back(d);
      }
  c->n_tiles = (int)t.size();
  cudaFree(c->tiles);
  c->tiles = nullptr;
  std::vector<TileDesc> th;
  half_tiles(t, th);
  c->n_tiles_half = (int)th.size();
  cudaFree(c->tiles_half);
  c->tiles_half = nullptr;
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->tiles_half, sizeof(TileDesc) * std::max<size_t>(1, th.size())));
  if (!th.empty())
    CUDA_OR_FAIL(c, cudaMemcpy(c->tiles_half, th.data(), sizeof(TileDesc) * th.size(),
                               cudaMemcpyHostToDevice));
  cudaFree(c->rec32);
  c->rec32 = nullptr;
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->tiles, sizeof(TileDesc) * std::max<size_t>(1, t.size())));
  if (!t.empty())
    CUDA_OR_FAIL(c, cudaMemcpy(c->tiles, t.data(), sizeof(TileDesc) * t.size(), cudaMemcpyHostToDevice));
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->rec32, sizeof(uint32_t) * rec32.size() + kGuardBytes));
  CUDA_OR_FAIL(c, cudaMemset(c->rec32, 0, sizeof(uint32_t) * rec32.size() + kGuardBytes));
  if (!rec32.empty())
    CUDA_OR_FAIL(c, cudaMemcpy(c->rec32, rec32.data(), sizeof(uint32_t) * rec32.size(),
                               cudaMemcpyHostToDevice));
  return LBM_OK;
}

extern "C" {

int lbm_create(lbm_ctx **out, int lattice, int nx, int ny, int nz, const double *s,
               int precision, double rho0) {
  if (!out) return fail(nullptr, LBM_EINVAL, "lbm_create: out is NULL");
  *out = nullptr;
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19 && lattice != LBM_D3Q15)
    return fail(nullptr, LBM_EINVAL, "lbm_create: unknown lattice %d", lattice);
  if (precision < LBM_F64 || precision > LBM_F16_DEV)
    return fail(nullptr, LBM_EINVAL, "lbm_create: unknown precision %d", precision);
  if (nx < 1 || ny < 1 || nz < 1)
    return fail(nullptr, LBM_EINVAL, "lbm_create: grid %dx%dx%d", nx, ny, nz);
  if (lattice == LBM_D2Q9 && nz != 1)
    return fail(nullptr, LBM_EINVAL, "lbm_create: D2Q9 needs nz == 1");
  if (!s) return fail(nullptr, LBM_EINVAL, "lbm_create: s is NULL");
  if (!(rho0 > 0) || !std::isfinite(rho0))
    return fail(nullptr, LBM_EINVAL, "lbm_create: rho0 must be > 0");
  const int Q = lattice == LBM_D2Q9 ? 9 : (lattice == LBM_D3Q15 ? 15 : 19);
  for (int k = 0; k < Q; ++k)
    if (!std::isfinite(s[k]) || s[k] < 0 || s[k] > 2)
      return fail(nullptr, LBM_EINVAL, "lbm_create: s[%d] = %g outside [0, 2]", k, s[k]);
  const long long N = (long long)nx * ny * nz;
  if (N > (1LL << 31) - 1) return fail(nullptr, LBM_EINVAL, "lbm_create: more than 2^31 nodes");

  lbm_ctx *c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(nullptr, LBM_ENOMEM, "lbm_create: host allocation");
  c->lattice = lattice; c->Q = Q; c->D = lattice == LBM_D2Q9 ? 2 : 3;
  c->precision = precision;
  c->nx = nx; c->ny = ny; c->nz = nz; c->N = N;
  c->rho0 = rho0;
  for (int k = 0; k < Q; ++k) c->s[k] = s[k];
  cudaError_t e = cudaGetDevice(&c->device);
  const size_t pop_bytes = pop_alloc_bytes(c);
  if (e == cudaSuccess) e = cudaMalloc(&c->pop_alloc, pop_bytes);
  if (e == cudaSuccess) c->pop = static_cast<char *>(c->pop_alloc) + kPopPadBytes;
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->cls, N + kGuardBytes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->pop_alloc, 0, pop_bytes);
  if (e == cudaSuccess) e = cudaMemset(c->cls, kFluid, N + kGuardBytes);
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
  if (e != cudaSuccess) {
    int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    fail(nullptr, code, "lbm_create: %s", cudaGetErrorString(e));
    lbm_destroy(c);
    return code;
  }
  c->n_fluid = N;
  c->geometry_set = true;  // all-fluid periodic box, no links
  if (upload_tiles(c, nullptr, nullptr, nullptr, nullptr) != LBM_OK) {
    g_create_error = c->err;
    lbm_destroy(c);
    return LBM_ECUDA;
  }
  refresh_args(c);
  *out = c;
  return LBM_OK;
}

int lbm_destroy(lbm_ctx *c) {
  if (!c) return LBM_OK;
  DeviceGuard dg(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->pop_alloc);
  cudaFree(c->cls);
  cudaFree(c->status);
  free_geometry(c);
  adj_ws_free(c);
  cudaFree(c->tiles);
  c->tiles = nullptr;
  cudaFree(c->tiles_half);
  c->tiles_half = nullptr;
  cudaFree(c->rec32);
  c->rec32 = nullptr;
  cudaFree(c->partials);
  cudaFree(c->norm_out);
  cudaFree(c->u_ref);
  cudaFree(c->u_prev);
  cudaFree(c->mom_rho);
  cudaFree(c->mom_u);
  delete c;
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx *c, void *stream) {
  if (!c) return LBM_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  return LBM_OK;
}

int lbm_set_skew(lbm_ctx *c, int sy, int sz) {
  if (!c) return LBM_EINVAL;
  if (sy < 0 || sy >= c->ny || sz < 0 || sz >= c->nz)
    return fail(c, LBM_EINVAL, "lbm_set_skew: need 0 <= sy < ny and 0 <= sz < nz");
  c->sy = sy;
  c->sz = sz;
  c->geometry_set = false;
  refresh_args(c);
  return LBM_OK;
}

int lbm_set_geometry(lbm_ctx *c, const uint8_t *solid, int64_t n_links, const int64_t *node,
                     const int32_t *dir, const double *q, const double *uw) {
  if (!c) return LBM_EINVAL;
  if (!solid) return fail(c, LBM_EINVAL, "lbm_set_geometry: solid is NULL");
  if (n_links < 0 || (n_links > 0 && (!node || !dir || !q)))
    return fail(c, LBM_EINVAL, "lbm_set_geometry: bad link arrays");
  DeviceGuard dg(c->device);
  const long long N = c->N;
  const int Q = c->Q;
  int rc = LBM_OK;
  std::vector<uint32_t> mask(N, 0);
  // every listed link: fluid node, solid neighbour, gamma in (0,1], no duplicate
  for (long long k = 0; k < n_links; ++k) {
    const long long n = node[k];
    const int d = dir[k];
    if (n < 0 || n >= N) return fail(c, LBM_EINVAL, "link %lld: node %lld out of range", k, n);
    if (d < 1 || d >= Q) return fail(c, LBM_EINVAL, "link %lld: direction %d out of range", k, d);
    if (solid[n]) return fail(c, LBM_EINVAL, "link %lld: node %lld is solid", k, n);
    if (!(q[k] > 0.0 && q[k] <= 1.0))
      return fail(c, LBM_EINVAL, "link %lld: wall fraction %g not in (0, 1]", k, q[k]);
    if (uw && !(std::isfinite(uw[3 * k]) && std::isfinite(uw[3 * k + 1]) &&
                std::isfinite(uw[3 * k + 2])))
      return fail(c, LBM_EINVAL, "link %lld: non-finite wall velocity", k);
    const int x = (int)(n % c->nx), y = (int)((n / c->nx) % c->ny), z = (int)(n / ((long long)c->nx * c->ny));
    long long nb = with_lat(c->lattice, [&](auto lat) {
      using L = decltype(lat);
      return wrap_host(c, x, y, z, L::ex(d), L::ey(d), L::ez(d));
    });
    if (!solid[nb])
      return fail(c, LBM_EINVAL, "link %lld: neighbour of node %lld along %d is fluid", k, n, d);
    if (mask[n] & (1u << d)) return fail(c, LBM_EINVAL, "link %lld: duplicate (%lld, %d)", k, n, d);
    mask[n] |= 1u << d;
  }
  // completeness: every fluid -> solid pair is listed (parallel over z-slabs)
  {
    const int nt = std::max(1, std::min<int>(std::thread::hardware_concurrency(), 32));
    std::vector<long long> bad(nt, -1);
    std::vector<std::thread> th;
    for (int w = 0; w < nt; ++w)
      th.emplace_back([&, w] {
        with_lat(c->lattice, [&](auto lat) {
          using L = decltype(lat);
          for (long long n = w; n < N; n += nt) {
            if (solid[n]) continue;
            const int x = (int)(n % c->nx), y = (int)((n / c->nx) % c->ny),
                      z = (int)(n / ((long long)c->nx * c->ny));
            for (int d = 1; d < L::Q; ++d) {
              const long long nb = wrap_host(c, x, y, z, L::ex(d), L::ey(d), L::ez(d));
              if (solid[nb] && !(mask[n] & (1u << d))) {
                bad[w] = n * 32 + d;
                return 0;
              }
            }
          }
          return 0;
        });
      });
    for (auto &t : th) t.join();
    for (long long v : bad)
      if (v >= 0)
        return fail(c, LBM_EINVAL, "no cut link listed for node %lld direction %lld (solid neighbour)",
                    v / 32, v % 32);
  }
  // convexity of the current scheme on every link (Eq. 2.12)
  for (long long k = 0; k < n_links; ++k) {
    const double l = l_of(c, q[k]);
    if (l < 0) return fail(c, LBM_EINVAL, "link %lld: l = %g < 0", k, l);
    if (!c->allow_nonconvex && !convex(q[k], l))
      return fail(c, LBM_ENONCONVEX, "link %lld: l = %g violates Eq. 2.12 at gamma = %g", k, l, q[k]);
  }
  // compaction: boundary records in node order, links in (node, d) order
  std::vector<uint8_t> cls(N);
  std::vector<int32_t> bidx(N, -1);
  std::vector<uint32_t> bmask;
  std::vector<int32_t> boff;
  long long nf = 0, off = 0;
  for (long long n = 0; n < N; ++n) {
    if (solid[n]) { cls[n] = kSolid; continue; }
    ++nf;
    if (mask[n]) {
      cls[n] = kBoundary;
      bidx[n] = (int32_t)bmask.size();
      bmask.push_back(mask[n]);
      boff.push_back((int32_t)off);
      off += __builtin_popcount(mask[n]);
    } else {
      cls[n] = kFluid;
    }
  }
  c->link_dir.assign(n_links, 0);
  c->link_node.assign(n_links, 0);
  c->link_q.assign(n_links, 0.0);
  c->link_uw.assign(3 * n_links, 0.0);
  c->link_src.assign(n_links, 0);
  for (long long k = 0; k < n_links; ++k) {
    const long long n = node[k];
    const int d = dir[k];
    const long long pos = boff[bidx[n]] + __builtin_popcount(mask[n] & ((1u << d) - 1u));
    c->link_dir[pos] = d;
    c->link_node[pos] = n;
    c->link_src[pos] = k;
    c->link_q[pos] = q[k];
    if (uw)
      for (int a = 0; a < 3; ++a) c->link_uw[3 * pos + a] = uw[3 * k + a];
  }
  // upload
  free_geometry(c);
  c->geometry_set = false;
  c->n_links = n_links;
  c->n_fluid = nf;
  c->n_boundary = (long long)bmask.size();
  const size_t cb = c->precision == LBM_F64 ? sizeof(double) : sizeof(float);
  CUDA_OR_FAIL(c, cudaMemcpy(c->cls, cls.data(), N, cudaMemcpyHostToDevice));
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->bidx, sizeof(int32_t) * N));
  CUDA_OR_FAIL(c, cudaMemcpy(c->bidx, bidx.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice));
  const size_t nb = std::max<size_t>(1, bmask.size());
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->bmask, sizeof(uint32_t) * nb));
  CUDA_OR_FAIL(c, cudaMalloc((void **)&c->boff, sizeof(int32_t) * nb));
  CUDA_OR_FAIL(c, cudaMalloc(&c->coef, 4 * cb * std::max<long long>(1, n_links)));
  CUDA_OR_FAIL(c, cudaMalloc(&c->lnk, link_bytes(c)));
  CUDA_OR_FAIL(c, cudaMemset(c->lnk, 0, link_bytes(c)));
  if (!bmask.empty()) {
    CUDA_OR_FAIL(c, cudaMemcpy(c->bmask, bmask.data(), sizeof(uint32_t) * bmask.size(),
                               cudaMemcpyHostToDevice));
    CUDA_OR_FAIL(c, cudaMemcpy(c->boff, boff.data(), sizeof(int32_t) * boff.size(),
                               cudaMemcpyHostToDevice));
  }
  if ((rc = upload_coefficients(c)) != LBM_OK) return rc;
  if ((rc = upload_tiles(c, solid, &cls, &bmask, &boff)) != LBM_OK) return rc;
  CUDA_OR_FAIL(c, cudaMemset(c->pop_alloc, 0, pop_alloc_bytes(c)));
  CUDA_OR_FAIL(c, cudaMemset(c->status, 0, sizeof(int)));
  cudaFree(c->u_prev);
  c->u_prev = nullptr;
  c->t = 0;
  ++c->state_serial;
  c->geometry_set = true;
  refresh_args(c);
  return build_two_node(c);
}

int lbm_set_two_node(lbm_ctx *c, int enable) {
  if (!c) return LBM_EINVAL;
  if (!c->geometry_set) return fail(c, LBM_ESTATE, "lbm_set_two_node: geometry not set");
  DeviceGuard dg(c->device);
  c->two_node = enable != 0;
  ++c->version;
  return build_two_node(c);
}

int lbm_set_scheme(lbm_ctx *c, double c0, double c1, double c2, double b, int allow_nonconvex) {
  if (!c) return LBM_EINVAL;
  if (!(std::isfinite(c0) && std::isfinite(c1) && std::isfinite(c2)))
    return fail(c, LBM_EINVAL, "lbm_set_scheme: non-finite l coefficients");
  if (!(b > 0.0 && b <= 1.0)) return fail(c, LBM_EINVAL, "lbm_set_scheme: b = %g not in (0, 1]", b);
  // l >= 0 on (0, 1]: check the ends and the vertex of the parabola
  auto lq = [&](double q) { return c0 + c1 * q + c2 * q * q; };
  double lmin = std::min(lq(1e-300), lq(1.0));
  if (c2 != 0.0) {
    const double v = -c1 / (2.0 * c2);
    if (v > 0.0 && v < 1.0) lmin = std::min(lmin, lq(v));
  }
  if (lmin < 0.0) return fail(c, LBM_EINVAL, "lbm_set_scheme: l < 0 for some gamma in (0, 1]");
  if (!allow_nonconvex)
    for (long long k = 0; k < c->n_links; ++k) {
      const double l = lq(c->link_q[k]);
      if (!convex(c->link_q[k], l))
        return fail(c, LBM_ENONCONVEX, "lbm_set_scheme: link %lld (gamma = %g) gets l = %g outside Eq. 2.12",
                    k, c->link_q[k], l);
    }
  c->c0 = c0; c->c1 = c1; c->c2 = c2; c->b = b;
  c->allow_nonconvex = allow_nonconvex != 0;
  DeviceGuard dg(c->device);
  int rc = upload_coefficients(c);
  refresh_args(c);
  return rc;
}

int lbm_set_wall_factor(lbm_ctx *c, double a0, double r) {
  if (!c) return LBM_EINVAL;
  if (!std::isfinite(a0) || !std::isfinite(r) || !(r > 0))
    return fail(c, LBM_EINVAL, "lbm_set_wall_factor: need finite a0 and r > 0");
  c->wf_a0 = a0;
  c->wf_r = r;
  c->wf_t0 = c->t;
  set_step_factor(c, c->t);
  ++c->version;   // batches take the factor of the member's time at each batch call
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx *c, int polls) {
  if (!c) return LBM_EINVAL;
  if (polls < 0) return fail(c, LBM_EINVAL, "lbm_set_wait_limit: polls = %d < 0", polls);
  c->wait_polls = polls;
  refresh_args(c);
  return LBM_OK;
}

int lbm_set_force(lbm_ctx *c, const double g[3]) {
  if (!c || !g) return LBM_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(g[k])) return fail(c, LBM_EINVAL, "lbm_set_force: non-finite force");
  for (int k = 0; k < 3; ++k) c->g[k] = (k < c->D) ? g[k] : 0.0;
  refresh_args(c);
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_ctx *c, const double *rho, const double *u) {
  if (!c) return LBM_EINVAL;
  if (!c->geometry_set) return fail(c, LBM_ESTATE, "lbm_init_equilibrium: geometry not set");
  DeviceGuard dg(c->device);
  // staging buffers are the context's moment buffers (same sizes), kept for reuse
  if (rho) {
    if (!c->mom_rho) CUDA_OR_FAIL(c, cudaMalloc(&c->mom_rho, sizeof(double) * c->N));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->mom_rho, rho, sizeof(double) * c->N, cudaMemcpyHostToDevice,
                                    c->stream));
  }
  if (u) {
    if (!c->mom_u) CUDA_OR_FAIL(c, cudaMalloc(&c->mom_u, sizeof(double) * c->N * c->D));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->mom_u, u, sizeof(double) * c->N * c->D,
                                    cudaMemcpyHostToDevice, c->stream));
  }
  CUDA_OR_FAIL(c, launch_init_equilibrium(c->lattice, c->precision, aux_args(c),
                                          rho ? c->mom_rho : nullptr, u ? c->mom_u : nullptr,
                                          c->stream));
  CUDA_OR_FAIL(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  c->t = 0;
  ++c->state_serial;
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx *c, const double *f) {
  if (!c || !f) return LBM_EINVAL;
  if (!c->geometry_set) return fail(c, LBM_ESTATE, "lbm_set_populations: geometry not set");
  DeviceGuard dg(c->device);
  double *df = nullptr;
  const size_t bytes = sizeof(double) * c->Q * c->N;
  CUDA_OR_FAIL(c, cudaMalloc(&df, bytes));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(df, f, bytes, cudaMemcpyHostToDevice, c->stream));
  CUDA_OR_FAIL(c, launch_set_populations(c->lattice, c->precision, aux_args(c), df, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  cudaFree(df);
  CUDA_OR_FAIL(c, cudaMemset(c->status, 0, sizeof(int)));
  c->t = 0;
  ++c->state_serial;
  return LBM_OK;
}

int lbm_get_populations(lbm_ctx *c, double *f) {
  if (!c || !f) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  double *df = nullptr;
  const size_t bytes = sizeof(double) * c->Q * c->N;
  CUDA_OR_FAIL(c, cudaMalloc(&df, bytes));
  CUDA_OR_FAIL(c, launch_get_populations(c->lattice, c->precision, aux_args(c), (c->t & 1) != 0,
                                         df, c->stream));
  CUDA_OR_FAIL(c, cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  cudaFree(df);
  return LBM_OK;
}

int lbm_step(lbm_ctx *c, int n) {
  if (!c) return LBM_EINVAL;
  if (n < 0) return fail(c, LBM_EINVAL, "lbm_step: n = %d < 0", n);
  if (!c->geometry_set) return fail(c, LBM_ESTATE, "lbm_step: geometry not set");
  DeviceGuard dg(c->device);
  for (int k = 0; k < n; ++k) {
    set_step_factor(c, c->t);
    const bool odd = (c->t & 1) != 0;
    cudaError_t e = cudaSuccess;
    if (c->n_tn)
      e = launch_two_node(c->lattice, c->precision, c->a64, c->a32, aux_args(c), odd, false, c->tn,
                          c->n_tn, c->tn_delta, c->stream);
    if (e == cudaSuccess)
      e = launch_sweep(c->lattice, c->precision, odd, c->a64, c->a32, c->tiles, c->n_tiles,
                       c->tiles_half, c->n_tiles_half, c->stream);
    if (e == cudaSuccess && c->n_tn)
      e = launch_two_node(c->lattice, c->precision, c->a64, c->a32, aux_args(c), odd, true, c->tn,
                          c->n_tn, c->tn_delta, c->stream);
    if (e != cudaSuccess) return fail(c, LBM_ECUDA, "lbm_step: %s", cudaGetErrorString(e));
    ++c->t;
    ++c->state_serial;
  }
  return LBM_OK;
}

int64_t lbm_time(const lbm_ctx *c) { return c ? c->t : -1; }

static int check_status(lbm_ctx *c) {
  int h = 0;
  CUDA_OR_FAIL(c, cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  if (h & 2) return fail(c, LBM_ETIMEOUT, "a sweep gave up waiting for a bulk copy (bounded wait)");
  if (h & 1) return fail(c, LBM_EDIVERGED, "a non-finite or runaway density was seen");
  return LBM_OK;
}

int lbm_moments_device(lbm_ctx *c, double *rho_dev, double *u_dev) {
  if (!c) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  CUDA_OR_FAIL(c, launch_moments(c->lattice, c->precision, aux_args(c), (c->t & 1) != 0, rho_dev,
                                 u_dev, c->stream));
  return LBM_OK;
}

int lbm_moments(lbm_ctx *c, double *rho, double *u) {
  if (!c) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  if (rho && !c->mom_rho) CUDA_OR_FAIL(c, cudaMalloc(&c->mom_rho, sizeof(double) * c->N));
  if (u && !c->mom_u) CUDA_OR_FAIL(c, cudaMalloc(&c->mom_u, sizeof(double) * c->N * c->D));
  int rc = lbm_moments_device(c, rho ? c->mom_rho : nullptr, u ? c->mom_u : nullptr);
  if (rc != LBM_OK) return rc;
  if (rho)
    CUDA_OR_FAIL(c, cudaMemcpyAsync(rho, c->mom_rho, sizeof(double) * c->N, cudaMemcpyDeviceToHost,
                                    c->stream));
  if (u)
    CUDA_OR_FAIL(c, cudaMemcpyAsync(u, c->mom_u, sizeof(double) * c->N * c->D,
                                    cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

int lbm_error_norms(lbm_ctx *c, const double *u_ref, lbm_norms *out) {
  if (!c || !out) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  const int nb = norm_blocks_for(c->N);
  if (!c->partials) CUDA_OR_FAIL(c, cudaMalloc(&c->partials, sizeof(double) * kNormFields * nb));
  if (!c->norm_out) CUDA_OR_FAIL(c, cudaMalloc(&c->norm_out, sizeof(double) * kNormFields));
  if (!c->u_prev) {
    CUDA_OR_FAIL(c, cudaMalloc(&c->u_prev, sizeof(double) * c->N * c->D));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->u_prev, 0, sizeof(double) * c->N * c->D, c->stream));
  }
  if (u_ref) {
    if (!c->u_ref) CUDA_OR_FAIL(c, cudaMalloc(&c->u_ref, sizeof(double) * c->N * c->D));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->u_ref, u_ref, sizeof(double) * c->N * c->D,
                                    cudaMemcpyHostToDevice, c->stream));
  }
  CUDA_OR_FAIL(c, launch_norm_partials(c->lattice, c->precision, aux_args(c), (c->t & 1) != 0,
                                       u_ref ? c->u_ref : nullptr, c->u_prev, c->partials, nb,
                                       c->stream));
  CUDA_OR_FAIL(c, launch_norm_finish(c->partials, nb, c->norm_out, c->stream));
  double h[kNormFields];
  CUDA_OR_FAIL(c, cudaMemcpyAsync(h, c->norm_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OR_FAIL(c, cudaStreamSynchronize(c->stream));
  const double nan = std::nan("");
  out->l2_rel = u_ref ? std::sqrt(h[0]) / std::sqrt(h[1]) : nan;
  out->linf = u_ref ? h[2] : nan;
  out->mass = h[3];
  out->mom[0] = h[4]; out->mom[1] = h[5]; out->mom[2] = h[6];
  out->residual = h[8] > 0 ? std::sqrt(h[7]) / std::sqrt(h[8]) : nan;
  if (h[9] > 0) return fail(c, LBM_EDIVERGED, "%g non-finite densities", h[9]);
  return check_status(c);
}

int lbm_error_norms_noalloc(lbm_ctx *c, const double *u_ref_dev, double *out_dev) {
  if (!c) return LBM_EINVAL;
  const char *why = "";
  const int rc = error_norms_noalloc(c->device, c->lattice, c->precision, aux_args(c),
                                     (c->t & 1) != 0, u_ref_dev, out_dev, c->stream, &why);
  if (rc != LBM_OK) return fail(c, rc, "lbm_error_norms_noalloc: %s", why);
  return LBM_OK;
}

int lbm_set_relaxation(lbm_ctx *c, const double *s) {
  if (!c || !s) return LBM_EINVAL;
  for (int k = 0; k < c->Q; ++k)
    if (!std::isfinite(s[k]) || s[k] < 0 || s[k] > 2)
      return fail(c, LBM_EINVAL, "lbm_set_relaxation: s[%d] = %g outside [0, 2]", k, s[k]);
  for (int k = 0; k < c->Q; ++k) c->s[k] = s[k];
  refresh_args(c);
  return LBM_OK;
}

int lbm_set_link_values(lbm_ctx *c, const double *q, const double *uw) {
  if (!c) return LBM_EINVAL;
  if (!c->geometry_set) return fail(c, LBM_ESTATE, "lbm_set_link_values: geometry not set");
  const long long nl = c->n_links;
  std::vector<double> nq(c->link_q), nuw(c->link_uw);
  for (long long pos = 0; pos < nl; ++pos) {
    const long long k = c->link_src[pos];
    if (q) {
      if (!(q[k] > 0.0 && q[k] <= 1.0))
        return fail(c, LBM_EINVAL, "lbm_set_link_values: link %lld: q = %g not in (0, 1]", k, q[k]);
      const double l = l_of(c, q[k]);
      if (l < 0) return fail(c, LBM_EINVAL, "lbm_set_link_values: link %lld: l < 0", k);
      if (!c->allow_nonconvex && !convex(q[k], l))
        return fail(c, LBM_ENONCONVEX, "lbm_set_link_values: link %lld: l = %g violates Eq. 2.12", k, l);
      nq[pos] = q[k];
    }
    if (uw)
      for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(uw[3 * k + a]))
          return fail(c, LBM_EINVAL, "lbm_set_link_values: link %lld: non-finite wall velocity", k);
        nuw[3 * pos + a] = uw[3 * k + a];
      }
  }
  c->link_q.swap(nq);
  c->link_uw.swap(nuw);
  DeviceGuard dg(c->device);
  const int rc = upload_coefficients(c);
  refresh_args(c);
  return rc;
}

// ---------------------------------------------------------------------------
// Discrete adjoint, split into a forward pass (checkpointed run and the loss) and
// a backward pass (recompute and adjoint sweep).  The tape between them lives in
// the context: the workspace buffers, the checkpoint times and the identity of
// the state the forward pass ended in.
// ---------------------------------------------------------------------------
namespace {
// workspace slots (lbm_ctx::adj_ws)
enum AdjSlot { kCk = 0, kSeg, kFin, kLam0, kLam1, kMask, kUt, kGs, kTot, kAcc, kDcoef, kJ, kGpart };

int adjoint_forward_impl(lbm_ctx *c, int n_steps, int checkpoint_every, const uint8_t *mask,
                         const double *u_target, double *loss) {
  c->tape.valid = false;
  if (n_steps < 1) return fail(c, LBM_EINVAL, "lbm_adjoint: n_steps >= 1");
  if (!mask || !u_target) return fail(c, LBM_EINVAL, "lbm_adjoint: mask and u_target are required");
  if (checkpoint_every < 0) return fail(c, LBM_EINVAL, "lbm_adjoint: checkpoint_every < 0");
  if (c->two_node)
    return fail(c, LBM_ESTATE, "lbm_adjoint: differentiates the single-node scheme; two-node is on");
  if (!c->geometry_set) return fail(c, LBM_ESTATE, "lbm_adjoint: geometry not set");
  const long long T = n_steps;
  long long K = checkpoint_every;
  if (K == 0) K = (long long)std::ceil(std::sqrt((double)T));
  if (K > T) K = T;
  const long long nseg = (T + K - 1) / K;
  const size_t csize = c->precision == LBM_F64 ? sizeof(double) : sizeof(float);
  const size_t state = (size_t)c->Q * c->N * csize;               // natural layout, compute type
  const size_t raw_pop = pop_alloc_bytes(c);
  const size_t raw_lnk = link_bytes(c);
  const long long nl1 = std::max<long long>(1, c->n_links);
  const bool natural = c->precision == LBM_F64 || c->precision == LBM_F32_DEV;
  const size_t ck_bytes = natural ? state : raw_pop + raw_lnk;
  char *ck = nullptr, *seg = nullptr, *fin = nullptr, *lam0 = nullptr, *lam1 = nullptr;
  uint8_t *dmask = nullptr;
  double *dut = nullptr, *dJ = nullptr;
  void *p = nullptr;
#define ADJ_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      c->a64.save = nullptr;                                                                \
      c->a32.save = nullptr;                                                                \
      adj_ws_free(c);                                                                       \
      return fail(c, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                  \
    }                                                                                       \
  } while (0)
  const long long pblocks = adjoint_partial_blocks(c->N);
  ADJ_CUDA(adj_ws_get(c, kCk, ck_bytes * nseg, (void **)&ck));
  ADJ_CUDA(adj_ws_get(c, kSeg, state * K, (void **)&seg));
  ADJ_CUDA(adj_ws_get(c, kFin, raw_pop + raw_lnk, (void **)&fin));
  ADJ_CUDA(adj_ws_get(c, kLam0, state, (void **)&lam0));
  ADJ_CUDA(adj_ws_get(c, kLam1, state, (void **)&lam1));
  ADJ_CUDA(adj_ws_get(c, kMask, c->N, (void **)&dmask));
  ADJ_CUDA(adj_ws_get(c, kUt, sizeof(double) * c->N * c->D, (void **)&dut));
  ADJ_CUDA(adj_ws_get(c, kGs, sizeof(double) * 19, &p));
  ADJ_CUDA(adj_ws_get(c, kTot, sizeof(double) * 2 * nl1, &p));
  ADJ_CUDA(adj_ws_get(c, kAcc, csize * 2 * nl1, &p));
  ADJ_CUDA(adj_ws_get(c, kDcoef, csize * 4 * nl1, &p));
  ADJ_CUDA(adj_ws_get(c, kJ, sizeof(double), (void **)&dJ));
  ADJ_CUDA(adj_ws_get(c, kGpart, sizeof(double) * c->Q * pblocks, &p));
  cudaStream_t st = c->stream;
  ADJ_CUDA(cudaMemcpyAsync(dmask, mask, c->N, cudaMemcpyHostToDevice, st));
  ADJ_CUDA(cudaMemcpyAsync(dut, u_target, sizeof(double) * c->N * c->D, cudaMemcpyHostToDevice, st));
  ADJ_CUDA(cudaMemsetAsync(dJ, 0, sizeof(double), st));
  AdjTape &tp = c->tape;
  tp.t0 = c->t;
  tp.T = T;
  tp.K = K;
  tp.nseg = nseg;
  tp.tck.assign(nseg, 0);
  // steps of a segment that also write each step's pre-collision state
  auto step_saving = [&](int len) -> int {
    for (int r = 0; r < len; ++r) {
      if (c->precision == LBM_F64) c->a64.save = reinterpret_cast<double *>(seg + state * r);
      else c->a32.save = reinterpret_cast<float *>(seg + state * r);
      const int e = lbm_step(c, 1);
      c->a64.save = nullptr;
      c->a32.save = nullptr;
      if (e != LBM_OK) return e;
    }
    return LBM_OK;
  };
  auto save_raw = [&](char *dst) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(dst, c->pop_alloc, raw_pop, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && c->lnk) e = cudaMemcpyAsync(dst + raw_pop, c->lnk, raw_lnk, cudaMemcpyDeviceToDevice, st);
    return e;
  };
  // FP64 and FP32 storage keep natural-layout checkpoints (the backward pass
  // recomputes with the push-form step); 16-bit storage keeps raw ones (it
  // recomputes with the sweep itself, so that its rounding matches this run).  The
  // last segment keeps its states as it goes, so the backward pass need not
  // recompute it.
  for (long long sgm = 0; sgm < nseg; ++sgm) {
    if (natural)
      ADJ_CUDA(launch_export_state(c->lattice, c->precision, aux_args(c), (c->t & 1) != 0,
                                   ck + ck_bytes * sgm, st));
    else
      ADJ_CUDA(save_raw(ck + ck_bytes * sgm));
    tp.tck[sgm] = c->t;
    const int len = (int)std::min(K, T - sgm * K);
    const int rc = sgm == nseg - 1 ? step_saving(len) : lbm_step(c, len);
    if (rc != LBM_OK) { adj_ws_free(c); return rc; }
  }
  ADJ_CUDA(save_raw(fin));
  // the loss (its kernel also writes lambda(T), which the backward pass recomputes)
  ADJ_CUDA(cudaMemsetAsync(lam1, 0, state, st));
  ADJ_CUDA(launch_export_state(c->lattice, c->precision, aux_args(c), (c->t & 1) != 0, lam1, st));
  ADJ_CUDA(launch_loss(c->lattice, c->precision, aux_args(c), lam1, dmask, dut, lam0, dJ, st));
  double hJ = 0.0;
  ADJ_CUDA(cudaMemcpyAsync(&hJ, dJ, sizeof(double), cudaMemcpyDeviceToHost, st));
  ADJ_CUDA(cudaStreamSynchronize(st));
  if (loss) *loss = hJ;
  const int rc = check_status(c);
  if (rc != LBM_OK) return rc;
  tp.version = c->version;
  tp.serial = c->state_serial;
  tp.valid = true;
  tp.last_saved = true;
  return LBM_OK;
}

int adjoint_backward_impl(lbm_ctx *c, double *grad_s, double *grad_q, double *grad_uw) {
  AdjTape &tp = c->tape;
  if (!tp.valid || tp.serial != c->state_serial || tp.version != c->version || c->t != tp.t0 + tp.T)
    return fail(c, LBM_ESTATE,
                "lbm_adjoint_backward: no forward pass for the current state (call "
                "lbm_adjoint_forward; stepping or changing the context in between discards it)");
  const long long T = tp.T, K = tp.K, nseg = tp.nseg;
  const size_t csize = c->precision == LBM_F64 ? sizeof(double) : sizeof(float);
  const size_t state = (size_t)c->Q * c->N * csize;
  const size_t raw_pop = pop_alloc_bytes(c);
  const size_t raw_lnk = link_bytes(c);
  const long long nl = c->n_links;
  const long long nl1 = std::max<long long>(1, nl);
  const bool natural = c->precision == LBM_F64 || c->precision == LBM_F32_DEV;
  const size_t ck_bytes = natural ? state : raw_pop + raw_lnk;
  const long long pblocks = adjoint_partial_blocks(c->N);
  char *ck = static_cast<char *>(c->adj_ws[kCk].first), *seg = static_cast<char *>(c->adj_ws[kSeg].first);
  char *fin = static_cast<char *>(c->adj_ws[kFin].first);
  char *lam0 = static_cast<char *>(c->adj_ws[kLam0].first), *lam1 = static_cast<char *>(c->adj_ws[kLam1].first);
  double *dgs = static_cast<double *>(c->adj_ws[kGs].first), *dtot = static_cast<double *>(c->adj_ws[kTot].first);
  void *acc = c->adj_ws[kAcc].first, *dcoef = c->adj_ws[kDcoef].first;
  double *gpart = static_cast<double *>(c->adj_ws[kGpart].first);
  cudaStream_t st = c->stream;
  tp.valid = false;   // reset below once the state is restored
  const uint8_t *dmask = static_cast<const uint8_t *>(c->adj_ws[kMask].first);
  const double *dut = static_cast<const double *>(c->adj_ws[kUt].first);
  double *dJ = static_cast<double *>(c->adj_ws[kJ].first);
  // lambda(T) from the forward end state (the current state): the state goes
  // through lam1, which the first adjoint step overwrites; solid entries of both
  // adjoint arrays stay zero
  ADJ_CUDA(cudaMemsetAsync(lam0, 0, state, st));
  ADJ_CUDA(cudaMemsetAsync(lam1, 0, state, st));
  ADJ_CUDA(cudaMemsetAsync(dJ, 0, sizeof(double), st));
  ADJ_CUDA(launch_export_state(c->lattice, c->precision, aux_args(c), (c->t & 1) != 0, lam1, st));
  ADJ_CUDA(launch_loss(c->lattice, c->precision, aux_args(c), lam1, dmask, dut, lam0, dJ, st));
  ADJ_CUDA(cudaMemsetAsync(gpart, 0, sizeof(double) * c->Q * pblocks, st));
  ADJ_CUDA(cudaMemsetAsync(dgs, 0, sizeof(double) * 19, st));
  ADJ_CUDA(cudaMemsetAsync(dtot, 0, sizeof(double) * 2 * nl1, st));
  ADJ_CUDA(cudaMemsetAsync(acc, 0, csize * 2 * nl1, st));
  // d(A, B, C)/dq per link (Eq. 2.10 with l = c0 + c1 q + c2 q^2), device order
  std::vector<double> hdc(4 * nl1, 0.0);
  for (long long k = 0; k < nl; ++k) {
    const double q = c->link_q[k], l = l_of(c, q), dl = c->c1 + 2.0 * c->c2 * q;
    const double inv2 = 1.0 / ((1.0 + l) * (1.0 + l));
    hdc[4 * k + 0] = (2.0 * q * dl - 2.0 * (1.0 + l)) * inv2;
    hdc[4 * k + 1] = dl * inv2;
    hdc[4 * k + 2] = (2.0 * (1.0 + l) - dl - 2.0 * q * dl) * inv2;
  }
  if (c->precision == LBM_F64) {
    ADJ_CUDA(cudaMemcpyAsync(dcoef, hdc.data(), sizeof(double) * hdc.size(), cudaMemcpyHostToDevice, st));
    ADJ_CUDA(cudaStreamSynchronize(st));     // hdc is about to go out of scope
  } else {
    std::vector<float> fdc(hdc.begin(), hdc.end());
    ADJ_CUDA(cudaMemcpyAsync(dcoef, fdc.data(), sizeof(float) * fdc.size(), cudaMemcpyHostToDevice, st));
    ADJ_CUDA(cudaStreamSynchronize(st));     // fdc is about to go out of scope
  }
  auto load_raw = [&](const char *src) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(c->pop_alloc, src, raw_pop, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && c->lnk) e = cudaMemcpyAsync(c->lnk, src + raw_pop, raw_lnk, cudaMemcpyDeviceToDevice, st);
    return e;
  };
  auto step_saving = [&](int len) -> int {
    for (int r = 0; r < len; ++r) {
      if (c->precision == LBM_F64) c->a64.save = reinterpret_cast<double *>(seg + state * r);
      else c->a32.save = reinterpret_cast<float *>(seg + state * r);
      const int e = lbm_step(c, 1);
      c->a64.save = nullptr;
      c->a32.save = nullptr;
      if (e != LBM_OK) return e;
    }
    return LBM_OK;
  };
  // backward pass: recompute each segment from its checkpoint (the last one only
  // when an earlier backward pass has overwritten the states the forward pass left),
  // then step back through it
  char *lin = lam0, *lout = lam1;
  const bool last_saved = tp.last_saved;
  tp.last_saved = false;          // the recomputation below reuses the segment buffer
  for (long long sgm = nseg - 1; sgm >= 0; --sgm) {
    const int len = (int)std::min(K, T - sgm * K);
    const bool saved = sgm == nseg - 1 && last_saved;
    // state of step r of this segment: the natural checkpoint itself for r = 0
    auto at = [&](int r) -> char * {
      return (natural && !saved && r == 0) ? ck + ck_bytes * sgm : seg + state * r;
    };
    if (!saved) {
      if (natural) {
        for (int r = 0; r + 1 < len; ++r) {
          set_step_factor(c, tp.tck[sgm] + r);
          ADJ_CUDA(launch_recompute_step(c->lattice, c->precision, c->a64, c->a32, aux_args(c),
                                         at(r), at(r + 1), st));
        }
      } else {
        ADJ_CUDA(load_raw(ck + ck_bytes * sgm));
        c->t = tp.tck[sgm];
        const int rc = step_saving(len);
        if (rc != LBM_OK) { adj_ws_free(c); return rc; }
      }
    }
    for (int r = len - 1; r >= 0; --r) {
      set_step_factor(c, tp.tck[sgm] + r);
      ADJ_CUDA(launch_adjoint_step(c->lattice, c->precision, c->a64, c->a32, aux_args(c), dcoef,
                                   acc, at(r), lin, lout, gpart, st));
      std::swap(lin, lout);
    }
    ADJ_CUDA(launch_link_flush(c->precision, acc, dtot, 2 * nl, st));
  }
  ADJ_CUDA(launch_adjoint_finish(c->lattice, gpart, pblocks, dgs, st));
  // back to the state after the forward run
  ADJ_CUDA(load_raw(fin));
  c->t = tp.t0 + T;
  std::vector<double> hgs(19), htot(2 * nl);
  ADJ_CUDA(cudaMemcpyAsync(hgs.data(), dgs, sizeof(double) * 19, cudaMemcpyDeviceToHost, st));
  if (nl)
    ADJ_CUDA(cudaMemcpyAsync(htot.data(), dtot, sizeof(double) * 2 * nl, cudaMemcpyDeviceToHost, st));
  ADJ_CUDA(cudaStreamSynchronize(st));
#undef ADJ_CUDA
  if (grad_s)
    for (int k = 0; k < c->Q; ++k) grad_s[k] = with_lat(c->lattice, [&](auto lat) {
      using L = decltype(lat);
      return L::conserved(k) ? 0.0 : hgs[k];
    });
  // fold in the q- and phi-dependent factors: W = 2 w_i rho0 e_i.phi / ((1 + l) c_s^2)
  // of Eq. 2.13 with c_s^2 = 1/3, so W' = -2 w_i rho0 3 e_i.phi l' / (1 + l)^2
  with_lat(c->lattice, [&](auto lat) {
    using L = decltype(lat);
    for (long long pos = 0; pos < nl; ++pos) {
      const long long k = c->link_src[pos];
      const int i = L::opp(c->link_dir[pos]);
      const double q = c->link_q[pos], l = l_of(c, q), dl = c->c1 + 2.0 * c->c2 * q;
      const double inv = 1.0 / (1.0 + l);
      const double ephi = L::ex(i) * c->link_uw[3 * pos] + L::ey(i) * c->link_uw[3 * pos + 1] +
                          L::ez(i) * c->link_uw[3 * pos + 2];
      const double wr = 2.0 * L::w(i) * c->rho0 * 3.0;
      const double dW = -wr * ephi * dl * inv * inv;
      const double s_lam = htot[2 * pos], s_q = htot[2 * pos + 1];
      if (grad_q) grad_q[k] = c->b * (s_q + dW * s_lam);
      if (grad_uw) {
        const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
        for (int a = 0; a < 3; ++a)
          grad_uw[3 * k + a] = (a < c->D) ? c->b * wr * inv * e[a] * s_lam : 0.0;
      }
    }
    return 0;
  });
  const int rc = check_status(c);
  if (rc != LBM_OK) return rc;
  // the state is the forward run's end state again: the tape stays usable
  tp.serial = c->state_serial;
  tp.valid = true;
  return LBM_OK;
}
}  // namespace

int lbm_adjoint_forward(lbm_ctx *c, int n_steps, int checkpoint_every, const uint8_t *mask,
                        const double *u_target, double *loss) {
  if (!c) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  return adjoint_forward_impl(c, n_steps, checkpoint_every, mask, u_target, loss);
}

int lbm_adjoint_backward(lbm_ctx *c, double *grad_s, double *grad_q, double *grad_uw) {
  if (!c) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  return adjoint_backward_impl(c, grad_s, grad_q, grad_uw);
}

int lbm_adjoint(lbm_ctx *c, int n_steps, int checkpoint_every, const uint8_t *mask,
                const double *u_target, double *loss, double *grad_s, double *grad_q,
                double *grad_uw) {
  if (!c) return LBM_EINVAL;
  DeviceGuard dg(c->device);
  int rc = adjoint_forward_impl(c, n_steps, checkpoint_every, mask, u_target, loss);
  if (rc == LBM_OK) rc = adjoint_backward_impl(c, grad_s, grad_q, grad_uw);
  return rc;
}

int lbm_query(const lbm_ctx *c, int *Q, int *D, int64_t *nodes, int64_t *fluid_nodes,
              int64_t *links) {
  if (!c) return LBM_EINVAL;
  if (Q) *Q = c->Q;
  if (D) *D = c->D;
  if (nodes) *nodes = c->N;
  if (fluid_nodes) *fluid_nodes = c->n_fluid;
  if (links) *links = c->n_links;
  return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many contexts advanced by one persistent launch per step, replayed
// from a CUDA graph.
// ---------------------------------------------------------------------------
// kernel classes of batch members: 2 * (rows aligned) + (skewed wrap); the general
// class (unaligned, skewed) serves every member
constexpr int kBatchClasses = 4;
constexpr int kBatchGeneral = 1;
struct BatchList {
  TileDesc *tiles = nullptr;
  int *tile_inst = nullptr;
  int n = 0;
};

struct lbm_batch {
  std::vector<lbm_ctx *> ctx;
  int lattice = 0, precision = 0, device = 0;
  cudaStream_t stream = nullptr;
  std::vector<std::vector<TileDesc>> host_tiles;   // per context
  std::vector<long long> versions;
  void *inst = nullptr;          // SweepArgs per context (compute type of the precision)
  BatchList lists[kBatchClasses];  // tile lists per kernel class (batch_upload)
  int n_tiles = 0;
  bool split = true;             // one launch per kernel class (lbm_batch_set_config)
  int tile_w = kTileW;           // nodes per tile in the lists: kTileW, or 32 (half tiles)
  bool big = false;
  int order = 1;                 // 0 context-major, 1 round-robin, 2 largest context first
  int blocks_per_sm = 0;         // 0: as many as fit
  cudaGraphExec_t graph = nullptr;
  bool graph_odd = false;        // parity of the first launch in the graph
  int graph_pairs = 0;           // even+odd launch pairs captured in the graph
  std::string err;
};

static int bfail(lbm_batch *b, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  else g_create_error = buf;
  return code;
}

#define BCUDA(b, call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                   #call, cudaGetErrorString(e_));                                      \
  } while (0)

static void batch_drop_graph(lbm_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_pairs = 0;
}

// Tile lists of the batch, one per kernel class, each in the batch's order.  A
// member's class is (rows start on 16-byte boundaries, skewed x-wrap); with the
// split on, each class runs the sweep specialised for it (aligned windows, no
// skew handling), otherwise -- and for grids whose slots need 64-bit indices --
// every member goes through the general kernel (unaligned windows, skew).
static bool member_aligned(const lbm_ctx *c) {
  return ((long long)c->nx * store_bytes(c->precision)) % 16 == 0;
}

static int batch_upload(lbm_batch *b) {
  const int n = (int)b->ctx.size();
  b->big = false;
  for (lbm_ctx *c : b->ctx)
    if ((long long)c->Q * slot_stride(c->N) >= (1LL << 31)) b->big = true;
  std::vector<int> cls_of(n, kBatchGeneral);
  if (b->split && !b->big)
    for (int k = 0; k < n; ++k) {
      const lbm_ctx *c = b->ctx[k];
      cls_of[k] = (member_aligned(c) ? 2 : 0) + ((c->sy != 0 || c->sz != 0) ? 1 : 0);
    }
  // the members' tiles in the batch's tile width (64-bit slot indices: 64 only)
  const bool halves = b->tile_w == 32 && !b->big;
  std::vector<std::vector<TileDesc>> halved(halves ? n : 0);
  for (int k = 0; k < (halves ? n : 0); ++k) half_tiles(b->host_tiles[k], halved[k]);
  const std::vector<std::vector<TileDesc>> &mt = halves ? halved : b->host_tiles;
  std::vector<int> ctx_order(n);
  for (int k = 0; k < n; ++k) ctx_order[k] = k;
  if (b->order == 2)
    std::stable_sort(ctx_order.begin(), ctx_order.end(), [&](int p, int q) {
      return mt[p].size() > mt[q].size();
    });
  b->n_tiles = 0;
  for (int cl = 0; cl < kBatchClasses; ++cl) {
    BatchList &bl = b->lists[cl];
    std::vector<TileDesc> t;
    std::vector<int> ti;
    if (b->order == 1) {
      // round-robin: one tile of every member of the class in turn
      std::vector<size_t> pos(n, 0);
      bool more = true;
      while (more) {
        more = false;
        for (int k : ctx_order)
          if (cls_of[k] == cl && pos[k] < mt[k].size()) {
            t.push_back(mt[k][pos[k]++]);
            ti.push_back(k);
            more = true;
          }
      }
    } else {
      for (int k : ctx_order)
        if (cls_of[k] == cl)
          for (const TileDesc &d : mt[k]) {
            t.push_back(d);
            ti.push_back(k);
          }
    }
    cudaFree(bl.tiles);
    cudaFree(bl.tile_inst);
    bl.tiles = nullptr;
    bl.tile_inst = nullptr;
    bl.n = (int)t.size();
    b->n_tiles += bl.n;
    if (t.empty()) continue;
    BCUDA(b, cudaMalloc((void **)&bl.tiles, sizeof(TileDesc) * t.size()));
    BCUDA(b, cudaMalloc((void **)&bl.tile_inst, sizeof(int) * ti.size()));
    BCUDA(b, cudaMemcpy(bl.tiles, t.data(), sizeof(TileDesc) * t.size(), cudaMemcpyHostToDevice));
    BCUDA(b, cudaMemcpy(bl.tile_inst, ti.data(), sizeof(int) * ti.size(), cudaMemcpyHostToDevice));
  }
  return LBM_OK;
}

static int batch_upload_args(lbm_batch *b) {
  const int n = (int)b->ctx.size();
  const bool f64 = b->precision == LBM_F64;
  const size_t one = f64 ? sizeof(SweepArgs<double>) : sizeof(SweepArgs<float>);
  std::vector<unsigned char> h(one * n);
  for (int k = 0; k < n; ++k) {
    lbm_ctx *c = b->ctx[k];
    std::memcpy(h.data() + one * k, f64 ? (const void *)&c->a64 : (const void *)&c->a32, one);
    b->versions[k] = c->version;
  }
  if (!b->inst) BCUDA(b, cudaMalloc(&b->inst, one * n));
  BCUDA(b, cudaMemcpy(b->inst, h.data(), one * n, cudaMemcpyHostToDevice));
  return LBM_OK;
}

static int batch_refresh_if_needed(lbm_batch *b) {
  bool stale = false;
  for (size_t k = 0; k < b->ctx.size(); ++k) stale |= b->ctx[k]->version != b->versions[k];
  if (!stale) return LBM_OK;
  // geometry may have changed: fetch the tile lists again
  for (size_t k = 0; k < b->ctx.size(); ++k) {
    lbm_ctx *c = b->ctx[k];
    b->host_tiles[k].resize(c->n_tiles);
    if (c->n_tiles)
      BCUDA(b, cudaMemcpy(b->host_tiles[k].data(), c->tiles, sizeof(TileDesc) * c->n_tiles,
                          cudaMemcpyDeviceToHost));
  }
  int rc = batch_upload(b);
  if (rc == LBM_OK) rc = batch_upload_args(b);
  batch_drop_graph(b);
  return rc;
}

static cudaError_t batch_launch(lbm_batch *b, bool odd, bool prepare_only) {
  for (int cl = 0; cl < kBatchClasses; ++cl) {
    const BatchList &bl = b->lists[cl];
    if (bl.n == 0) continue;
    const bool aligned = (cl & 2) != 0, skew = (cl & 1) != 0;
    cudaError_t e;
    switch (b->lattice) {
      case LBM_D2Q9:
        e = launch_sweep_batch_d2q9(b->precision, b->big ? kTileW : b->tile_w, odd, b->inst, bl.tiles, bl.tile_inst, bl.n, b->big,
                                    aligned, skew, b->blocks_per_sm, b->stream, prepare_only);
        break;
      case LBM_D3Q15:
        e = launch_sweep_batch_d3q15(b->precision, b->big ? kTileW : b->tile_w, odd, b->inst, bl.tiles, bl.tile_inst, bl.n, b->big,
                                     aligned, skew, b->blocks_per_sm, b->stream, prepare_only);
        break;
      default:
        e = launch_sweep_batch_d3q19(b->precision, b->big ? kTileW : b->tile_w, odd, b->inst, bl.tiles, bl.tile_inst, bl.n, b->big,
                                     aligned, skew, b->blocks_per_sm, b->stream, prepare_only);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static int batch_check_parity(lbm_batch *b, bool *odd) {
  const long long t0 = b->ctx[0]->t;
  for (lbm_ctx *c : b->ctx) {
    if (!c->geometry_set) return bfail(b, LBM_ESTATE, "a context of the batch has no geometry");
    if (c->two_node) return bfail(b, LBM_ESTATE, "batches run the single-node scheme; a member has two-node on");
    if ((c->t & 1) != (t0 & 1))
      return bfail(b, LBM_ESTATE, "contexts of a batch must be at the same time parity");
  }
  *odd = (t0 & 1) != 0;
  return LBM_OK;
}

static int batch_run_plain(lbm_batch *b, int n) {
  bool odd;
  int rc = batch_check_parity(b, &odd);
  if (rc != LBM_OK) return rc;
  for (int k = 0; k < n; ++k) {
    BCUDA(b, batch_launch(b, ((k & 1) != 0) != odd, false));
  }
  for (lbm_ctx *c : b->ctx) {
    c->t += n;
    c->state_serial += n;
  }
  return LBM_OK;
}

extern "C" {

int lbm_batch_create(lbm_batch **out, int n, lbm_ctx *const *ctxs) {
  if (!out) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: out is NULL");
  *out = nullptr;
  if (n < 1 || !ctxs) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: empty batch");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d is NULL", k);
    if (ctxs[k]->lattice != ctxs[0]->lattice || ctxs[k]->precision != ctxs[0]->precision ||
        ctxs[k]->device != ctxs[0]->device)
      return bfail(nullptr, LBM_EINVAL,
                   "lbm_batch_create: contexts must share lattice, precision and device");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d repeated", k);
  }
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ENOMEM, "lbm_batch_create: host allocation");
  b->ctx.assign(ctxs, ctxs + n);
  b->lattice = ctxs[0]->lattice;
  b->precision = ctxs[0]->precision;
  b->device = ctxs[0]->device;
  b->stream = ctxs[0]->stream;
  b->host_tiles.resize(n);
  b->versions.assign(n, -1);
  DeviceGuard dg(b->device);
  const int rc = batch_refresh_if_needed(b);
  if (rc != LBM_OK) {
    g_create_error = b->err;
    lbm_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch *b) {
  if (!b) return LBM_OK;
  DeviceGuard dg(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  cudaFree(b->inst);
  for (BatchList &bl : b->lists) {
    cudaFree(bl.tiles);
    cudaFree(bl.tile_inst);
  }
  delete b;
  return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch *b, void *stream) {
  if (!b) return LBM_EINVAL;
  b->stream = static_cast<cudaStream_t>(stream);
  batch_drop_graph(b);
  return LBM_OK;
}

int lbm_batch_set_config(lbm_batch *b, int order, int blocks_per_sm, int split, int tile_w) {
  if (!b) return LBM_EINVAL;
  if (order < 0 || order > 2 || blocks_per_sm < 0 || blocks_per_sm > 32 || split < 0 || split > 1 ||
      (tile_w != 32 && tile_w != 64))
    return bfail(b, LBM_EINVAL,
                 "lbm_batch_set_config: order in 0..2, blocks_per_sm in 0..32, split 0 or 1, "
                 "tile_w 32 or 64");
  DeviceGuard dg(b->device);
  b->order = order;
  b->blocks_per_sm = blocks_per_sm;
  b->split = split != 0;
  b->tile_w = tile_w;
  batch_drop_graph(b);
  return batch_upload(b);
}

int lbm_batch_step(lbm_batch *b, int n) {
  if (!b) return LBM_EINVAL;
  if (n < 0) return bfail(b, LBM_EINVAL, "lbm_batch_step: n < 0");
  DeviceGuard dg(b->device);
  int rc = batch_refresh_if_needed(b);
  if (rc != LBM_OK) return rc;
  bool odd;
  if ((rc = batch_check_parity(b, &odd)) != LBM_OK) return rc;
  if (n < 2) return batch_run_plain(b, n);
  // a graph of one even+odd pair of launches starting at the current parity
  if (!b->graph || b->graph_odd != odd) {
    batch_drop_graph(b);
    BCUDA(b, batch_launch(b, odd, true));    // launch attributes before the capture
    BCUDA(b, batch_launch(b, !odd, true));
    cudaStream_t cap = b->stream;
    bool own = false;
    if (cap == nullptr) {  // the legacy stream cannot be captured: use a private one
      BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      own = true;
    }
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    cudaStream_t saved = b->stream;
    b->stream = cap;
    cudaError_t e1 = batch_launch(b, odd, false);
    cudaError_t e2 = batch_launch(b, !odd, false);
    b->stream = saved;
    cudaError_t e3 = cudaStreamEndCapture(cap, &g);
    if (own) cudaStreamDestroy(cap);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(b, LBM_ECUDA, "lbm_batch_step: graph capture failed: %s",
                   cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
    }
    cudaError_t e4 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, LBM_ECUDA, "lbm_batch_step: %s", cudaGetErrorString(e4));
    }
    b->graph_odd = odd;
    b->graph_pairs = 1;
  }
  for (int k = 0; k + 1 < n; k += 2) BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  for (lbm_ctx *c : b->ctx) {
    c->t += n - (n & 1);
    c->state_serial += n - (n & 1);
  }
  if (n & 1) return batch_run_plain(b, 1);
  return LBM_OK;
}

int lbm_batch_tune(lbm_batch *b, int trial_steps, int *order_out, int *blocks_out, int *split_out,
                   int *tile_w_out) {
  if (!b) return LBM_EINVAL;
  if (trial_steps < 2) return bfail(b, LBM_EINVAL, "lbm_batch_tune: trial_steps >= 2");
  trial_steps &= ~1;
  DeviceGuard dg(b->device);
  int rc = batch_refresh_if_needed(b);
  if (rc != LBM_OK) return rc;
  bool odd;
  if ((rc = batch_check_parity(b, &odd)) != LBM_OK) return rc;
  // snapshot populations and link buffers: tuning leaves the state untouched
  size_t bytes = 0;
  for (lbm_ctx *c : b->ctx)
    bytes += pop_alloc_bytes(c) + link_bytes(c);
  void *snap = nullptr;
  BCUDA(b, cudaMalloc(&snap, bytes));
  auto copy_state = [&](bool save) -> cudaError_t {
    size_t o = 0;
    for (lbm_ctx *c : b->ctx) {
      const size_t pb = pop_alloc_bytes(c);
      const size_t lb = link_bytes(c);
      char *s = static_cast<char *>(snap) + o;
      cudaError_t e = save ? cudaMemcpyAsync(s, c->pop_alloc, pb, cudaMemcpyDeviceToDevice, b->stream)
                           : cudaMemcpyAsync(c->pop_alloc, s, pb, cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
      if (c->lnk) {
        e = save ? cudaMemcpyAsync(s + pb, c->lnk, lb, cudaMemcpyDeviceToDevice, b->stream)
                 : cudaMemcpyAsync(c->lnk, s + pb, lb, cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return e;
      }
      o += pb + lb;
    }
    return cudaSuccess;
  };
  cudaError_t e = copy_state(true);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int orders[3] = {0, 1, 2};
  const int blocks[3] = {0, 4, 3};
  const int widths[2] = {kTileW, 32};
  float best = 1e30f;
  int best_o = b->order, best_b = b->blocks_per_sm, best_w = b->tile_w;
  bool best_s = b->split;
  for (int wi = 0; wi < (b->big ? 1 : 2) && e == cudaSuccess && rc == LBM_OK; ++wi)
  for (int si = 0; si < 2 && e == cudaSuccess && rc == LBM_OK; ++si)
  for (int oi = 0; oi < 3 && e == cudaSuccess && rc == LBM_OK; ++oi)
    for (int bi = 0; bi < 3 && e == cudaSuccess; ++bi) {
      b->tile_w = widths[wi];
      b->split = si == 0;
      b->order = orders[oi];
      b->blocks_per_sm = blocks[bi];
      if ((rc = batch_upload(b)) != LBM_OK) break;
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = batch_launch(b, (k & 1) != odd, false);  // warm
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = batch_launch(b, (k & 1) != odd, false);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_o = orders[oi];
        best_b = blocks[bi];
        best_s = b->split;
        best_w = b->tile_w;
      }
      if (e == cudaSuccess) e = copy_state(false);
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(snap);
  if (rc != LBM_OK) return rc;
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_tune: %s", cudaGetErrorString(e));
  b->order = best_o;
  b->blocks_per_sm = best_b;
  b->split = best_s;
  b->tile_w = best_w;
  batch_drop_graph(b);
  if ((rc = batch_upload(b)) != LBM_OK) return rc;
  if (order_out) *order_out = best_o;
  if (blocks_out) *blocks_out = best_b;
  if (split_out) *split_out = best_s ? 1 : 0;
  if (tile_w_out) *tile_w_out = best_w;
  return LBM_OK;
}

int lbm_batch_query(const lbm_batch *b, int *n_contexts, int64_t *tiles, int *order,
                    int *blocks_per_sm, int *launches_per_step, int *tile_w) {
  if (!b) return LBM_EINVAL;
  if (n_contexts) *n_contexts = (int)b->ctx.size();
  if (tiles) *tiles = b->n_tiles;
  if (order) *order = b->order;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (launches_per_step) {
    int k = 0;
    for (const BatchList &bl : b->lists) k += bl.n > 0 ? 1 : 0;
    *launches_per_step = k;
  }
  if (tile_w) *tile_w = b->big ? kTileW : b->tile_w;
  return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) {
  return b ? b->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
