// lbm_internal.h -- device argument blocks and launcher declarations shared by the
// library's translation units (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace lbm {

// Makes `dev` the current device for the lifetime of the object and restores the
// caller's current device afterwards: entry points run on their context's device
// without leaving the calling thread's device changed.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard &) = delete;
  DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// Tile width of the sweep: a warp handles kTileW consecutive nodes along x,
// kNodesPerLane per lane.
#ifndef LBM_NPL
#define LBM_NPL 2
#endif
constexpr int kNodesPerLane = LBM_NPL;
constexpr int kTileW = 32 * kNodesPerLane;

static_assert(kTileW <= 64, "tile lane masks are 64-bit");

// One unit of sweep work: kTileW consecutive nodes (x0 .. x0+kTileW-1) of row
// (y, z) = (yz & 0xffff, yz >> 16) holding at least one fluid node.  Bit k of
// solid is set when node x0+k is solid or lies beyond the row; bit k of bnd when
// it is a boundary node.  The tile's boundary records are rec32[rb ...] in node
// order, and its cut links start at link lb.
struct alignas(16) TileDesc {
  int x0, yz, rb, lb;
  unsigned long long solid, bnd;
};
// packed record of a boundary node: cut-direction mask in bits 0..18, offset of
// its first link relative to the tile's lb in bits 19..31
constexpr int kRecShift = 19;

// node classes stored one byte per node
enum : uint8_t { kFluid = 0, kBoundary = 1, kSolid = 2 };

// Geometry on the device.  Boundary nodes (fluid nodes with at least one cut link)
// own a record b = bidx[n]: bmask[b] has bit d set when x_n + e_d is solid, and the
// node's links occupy coef[boff[b] .. boff[b] + popcount(bmask[b]) - 1] in
// ascending d.  rec32[b] holds the same record packed relative to its tile, for
// the sweep's bulk copies; records are numbered in node order, so the records of
// one tile are contiguous.  rec32 is allocated with guard bytes after its end.
struct DevGeometry {
  const uint8_t *cls = nullptr;
  const int32_t *bidx = nullptr;
  const uint32_t *bmask = nullptr;
  const int32_t *boff = nullptr;
  const uint32_t *rec32 = nullptr; // packed records (see TileDesc), in node order
  const void *coef = nullptr;      // 4 coefficients per link, compute type
  void *lnk = nullptr;             // one storage element per link (see below)
};

// The link buffer carries, from an even step to the following odd step, the value
// f_i(x_f, t+1) the boundary scheme produced for each cut link (i = opp(d)).  The
// odd step reads it where the plain AA pattern would read slot d of the solid
// neighbour x_f + e_d, so solid nodes' slots are never written or needed.

// Per-link coefficients of Eq. 2.13 with b folded in: the new value of the
// population i = opp(d) is (1-b) g_i + a g_d + bb g'_i + c g'_d + w.
template <class C>
struct alignas(4 * sizeof(C)) LinkCoef {
  C a, bb, c, w;
};

// Populations: Q slots of S >= N storage elements each (S a multiple of 64),
// population i of node n at pop[i*S + n].  The allocation extends kPopPadBytes
// before pop and after the last slot, so that aligned bulk copies of a row window
// may start a little before a row or end a little after it.
constexpr long long kPopPadBytes = 4096;
inline long long slot_stride(long long N) { return (N + 63) / 64 * 64; }

// default number of barrier polls before a sweep gives up waiting for a copy
// (each poll suspends for at most 1 ms: about 1 s in all)
constexpr int kWaitLimitDefault = 1000;

template <class C>
struct SweepArgs {
  void *pop;                 // population i of node n at pop[i*S + n]
  long long N;               // nodes
  long long S;               // slot stride
  int nx, ny, nz, sy, sz;
  DevGeometry geo;
  C sn[19];                  // s_k / |M_k|^2 for the non-conserved rows
  C F[3];                    // rho0 g / |M_j|^2
  C inv_rho0;
  C one_minus_b;
  C wfac;                    // factor on every link's wall velocity in this step
  int *status;               // bit 0: non-finite density seen, bit 1: bounded wait gave up
  int wait_polls;            // polls of a tile's barrier before the sweep gives up
  // element offsets of the stores of an interior node: even step slot opp(i) of
  // the node itself, odd step slot i of x + e_i (no wrap)
  long long koff_even[19];
  long long koff_odd[19];
  // the odd-step store of node (0, y, z) across the x-wrap lands at koff_odd[i] +
  // kwrap, that of node (nx-1, y, z) at koff_odd[i] - kwrap, when the skew-shifted
  // rows stay inside the grid: kwrap = nx (1 + sy) + nx ny sz
  long long kwrap;
  // when non-null, the sweep also writes every fluid node's pre-collision
  // deviations g_i(x, t) here, natural layout save[i*N + n] (adjoint recomputation)
  C *save = nullptr;
};

// launchers (return cudaGetLastError() of the launch)
// tiles: the 64-node tile list; tiles_half: the same tiles cut into 32-node halves
// (used by the storage types whose single-context sweep runs half tiles)
cudaError_t launch_sweep(int lattice, int precision, bool odd, const SweepArgs<double> &a64,
                         const SweepArgs<float> &a32, const TileDesc *tiles, int n_tiles,
                         const TileDesc *tiles_half, int n_half, cudaStream_t st);

struct AuxArgs {
  void *pop;
  long long N;               // nodes
  long long S;               // slot stride
  int nx, ny, nz, sy, sz;
  const uint8_t *cls;
  const int32_t *bidx;       // boundary records and link buffer (odd-time reads)
  const uint32_t *bmask;
  const int32_t *boff;
  const void *lnk;
  double rho0;
  double g[3];
};

// f = f^eq(rho, u) (deviation form) in the even-time layout; rho/u device or null
cudaError_t launch_init_equilibrium(int lattice, int precision, const AuxArgs &a,
                                    const double *rho, const double *u, cudaStream_t st);
// full populations f[i*N+n] (double, device) <-> storage at time parity `odd`
cudaError_t launch_get_populations(int lattice, int precision, const AuxArgs &a, bool odd,
                                   double *f, cudaStream_t st);
cudaError_t launch_set_populations(int lattice, int precision, const AuxArgs &a,
                                   const double *f, cudaStream_t st);
// rho (N) and u (D*N) in FP64 on the device; null pointers skip that output
cudaError_t launch_moments(int lattice, int precision, const AuxArgs &a, bool odd, double *rho,
                           double *u, cudaStream_t st);

// Block partial sums of the error norms.  Layout of one partial record (doubles):
// [0] sum |u_ref-u|^2, [1] sum |u_ref|^2, [2] max |u_ref-u|, [3] sum rho,
// [4..6] sum j, [7] sum |u - u_prev|^2, [8] sum |u|^2, [9] non-finite count
constexpr int kNormFields = 10;
cudaError_t launch_norm_partials(int lattice, int precision, const AuxArgs &a, bool odd,
                                 const double *u_ref, double *u_prev, double *partials,
                                 int n_blocks, cudaStream_t st);
cudaError_t launch_norm_finish(const double *partials, int n_blocks, double *out,
                               cudaStream_t st);

// adjoint (adjoint.cu); compute type double for precision 0, float otherwise
cudaError_t launch_export_state(int lattice, int precision, const AuxArgs &a, bool odd, void *out,
                                cudaStream_t st);
cudaError_t launch_import_state(int lattice, int precision, const AuxArgs &a, const void *in,
                                cudaStream_t st);
cudaError_t launch_loss(int lattice, int precision, const AuxArgs &a, const void *g,
                        const uint8_t *mask, const double *u_target, void *lam, double *J,
                        cudaStream_t st);
// a cut link that takes the two-node scheme (Eq. 2.11): boundary node x_f, its
// fluid neighbour x_l = x_f + e_i behind it, link index k, wall direction d
struct TwoNodeLink {
  long long xf, xl;
  int k, d;
};
// pre (post = false): difference of the two schemes for every listed link into
// delta, from the state at time t (parity odd); post: add it to the values the
// step t -> t+1 wrote
cudaError_t launch_two_node(int lattice, int precision, const SweepArgs<double> &a64,
                            const SweepArgs<float> &a32, const AuxArgs &a, bool odd, bool post,
                            const TwoNodeLink *tn, long long n_tn, void *delta, cudaStream_t st);

// one step of the adjoint sweep: lambda(t) from lambda(t+1) and the pre-collision
// state f (natural layout, compute type); per-link sums into link_acc (2 compute-type
// values per link), dJ/ds into the per-block partial records
cudaError_t launch_adjoint_step(int lattice, int precision, const SweepArgs<double> &a64,
                                const SweepArgs<float> &a32, const AuxArgs &a, const void *dcoef,
                                void *link_acc, const void *f, const void *lam_in, void *lam_out,
                                double *gs_part, cudaStream_t st);
// f(t+1) from f(t), both natural layout in the compute type (push form, same
// arithmetic as the sweep); for recomputing adjoint segments of FP64 / FP32 storage
cudaError_t launch_recompute_step(int lattice, int precision, const SweepArgs<double> &a64,
                                  const SweepArgs<float> &a32, const AuxArgs &a, const void *fin,
                                  void *fout, cudaStream_t st);
// tot[j] += link_acc[j], link_acc[j] = 0 for j < n
cudaError_t launch_link_flush(int precision, void *link_acc, double *tot, long long n,
                              cudaStream_t st);
// per-block partial sums of dJ/ds (Q doubles per block), reduced by launch_adjoint_finish
long long adjoint_partial_blocks(long long N);
cudaError_t launch_adjoint_finish(int lattice, const double *gs_part, long long n_blocks,
                                  double *grad_s, cudaStream_t st);
int norm_blocks_for(long long N);

}  // namespace lbm
