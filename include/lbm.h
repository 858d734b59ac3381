/*
 * lbm.h -- C-ABI of the GB300 lattice-Boltzmann library with the single-node
 * second-order boundary schemes of Zhao & Yong, "A family of single-node
 * second-order boundary schemes for the lattice Boltzmann method"
 * (arXiv:1712.08288).
 *
 * What one step computes (lbm_step):
 *   - collision, point-wise, MRT form  f' = f - M^-1 S M (f - f^eq)   (Eq. 2.2a;
 *     Appendix), incompressible equilibrium of Eq. 42 with rho0 u = sum c_i f_i;
 *   - body force: rho0*g added to the momentum moments after relaxation
 *     (the paper uses a force, Sec. 3, but states no forcing scheme; this is the
 *     library's reading, and the velocity it reports is u = j/rho0 + g/2);
 *   - advection f_i(x + e_i, t+1) = f'_i(x, t) between fluid nodes (Eq. 2.2b);
 *   - for every cut link the single-node boundary value (Eqs. 2.10 and 2.13):
 *       f_i(x_f,t+1) = (1-b) f_i(x_f,t) + b [ (1+l-2g)/(1+l) f_ib(x_f,t)
 *                      + l/(1+l) f'_i(x_f,t) + (2g-l)/(1+l) f'_ib(x_f,t)
 *                      + 2/(1+l) w_i rho0 (e_i . phi(x_b)) / c_s^2 ]
 *     with g = gamma = the link's wall fraction, ib the opposite of i, and
 *     l = c0 + c1 g + c2 g^2 (the family parameter of Sec. 2; the five rules of
 *     Sec. 3 are (0,1,0), (0,1.5,0), (0,2,0), (0,0,1), (0,1,1)).
 *   Lattice units: h = delta_t = c = 1, c_s^2 = 1/3.
 *
 * Lattices and numbering:
 *   LBM_D2Q9  directions 0..8 in the paper's Appendix order
 *             (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1);
 *             moments (rows of M, the Appendix matrix): rho, e, eps, j_x, q_x,
 *             j_y, q_y, p_xx, p_xy.
 *   LBM_D3Q19 (not in the paper; the 3D MRT family it cites, d'Humieres et al.
 *             2002) directions 0..18: rest; +x,-x,+y,-y,+z,-z; (1,1,0),(-1,-1,0),
 *             (1,-1,0),(-1,1,0), (1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1), (0,1,1),
 *             (0,-1,-1),(0,1,-1),(0,-1,1); moments rho, e, eps, j_x, q_x, j_y,
 *             q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x,
 *             m_y, m_z.
 *   LBM_D3Q15 directions 0..14 in the paper's Appendix order: rest; +x,-x,+y,-y,
 *             +z,-z; (1,1,1),(-1,1,1),(1,-1,1),(-1,-1,1),(1,1,-1),(-1,1,-1),
 *             (1,-1,-1),(-1,-1,-1); moments (the Appendix matrix): rho, e, eps,
 *             j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, p_ww, p_xy, p_yz, p_xz, m_xyz.
 *
 * Grid: nx*ny*nz nodes (nz = 1 for D2Q9), node index n = x + nx*(y + ny*z).
 *   Every axis is periodic; the x-wrap may be skewed (lbm_set_skew).  Walls that
 *   are not periodic are expressed with solid nodes: a fluid node's every
 *   neighbour is either fluid or a solid node with a cut link toward it.
 *
 * Conventions for every call:
 *   - Host pointers are borrowed for the duration of the call and copied; the
 *     caller keeps ownership.  "_device" calls take device pointers that the
 *     caller owns (e.g. from PyTorch); the library never frees them.
 *   - Every call returns an lbm_status and records a message readable with
 *     lbm_last_error().  Nothing throws across the ABI.
 *   - A context is not thread-safe.  Work is issued on the context's stream
 *     (lbm_set_stream; default: the legacy default stream).  Calls that return
 *     host data synchronise that stream.
 *   - Device memory (populations, geometry) is allocated by the library with
 *     cudaMalloc on the device current at lbm_create, and freed by lbm_destroy.
 *   - Every call that touches the GPU makes its context's (or batch's) device
 *     current for its duration and restores the calling thread's current device
 *     before it returns.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q15 = 2 };

/* Storage precision of the populations.  F64 stores and computes in double.
 * The _DEV variants store deviations g_i = f_i - w_i rho0 (the scheme is exact in
 * that form: its coefficients sum to one and the equilibrium is linear in rho) and
 * compute in float. */
enum lbm_precision { LBM_F64 = 0, LBM_F32_DEV = 1, LBM_BF16_DEV = 2, LBM_F16_DEV = 3 };

enum lbm_status {
  LBM_OK = 0,
  LBM_EINVAL = -1,      /* bad argument (message says which)                      */
  LBM_ENOMEM = -2,      /* device or host allocation failed                       */
  LBM_ECUDA = -3,       /* a CUDA call failed (message carries cudaGetErrorString) */
  LBM_ENONCONVEX = -4,  /* a link's l violates Eq. 2.12 and nonconvex not allowed  */
  LBM_EDIVERGED = -5,   /* a non-finite or runaway density was seen               */
  LBM_ETIMEOUT = -6,    /* a bounded device wait gave up                          */
  LBM_ESTATE = -7       /* call out of order (e.g. lbm_step before lbm_set_geometry) */
};

/* Create a context on the current CUDA device.
 *   lattice   LBM_D2Q9, LBM_D3Q19 or LBM_D3Q15; nz must be 1 for D2Q9.
 *   nx,ny,nz  grid size, each >= 1 (one- and two-node extents are periodic like
 *             any other: a node may be its own neighbour across the wrap).
 *   s         Q relaxation rates in the moment order above (diagonal of S,
 *             Appendix); the rates of rho and j have no effect (conserved).
 *   precision an lbm_precision.
 *   rho0      the mean density rho0 of Eq. 42 (> 0).
 * Populations start at rest (f = w_i rho0); the geometry starts all-fluid; the
 * scheme starts at l = gamma, b = 1 (Remark 4's special case); no force. */
int lbm_create(lbm_ctx **out, int lattice, int nx, int ny, int nz,
               const double *s, int precision, double rho0);
int lbm_destroy(lbm_ctx *ctx);

/* Stream on which all later work is issued (a cudaStream_t; NULL = legacy). */
int lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* Skewed x-periodicity: the field is invariant under the translation
 * (nx, sy, sz); 0 <= sy < ny, 0 <= sz < nz.  Invalidates the geometry (call
 * lbm_set_geometry again). */
int lbm_set_skew(lbm_ctx *ctx, int sy, int sz);

/* Geometry and cut links (Sec. 2, Fig. 1).
 *   solid    nodes bytes, nonzero = solid (outside the fluid).
 *   n_links  number of cut links.
 *   node[k]  fluid node x_f of link k.
 *   dir[k]   direction d pointing from x_f toward the wall: x_f + e_d is solid.
 *            The population the scheme computes is i = opposite(d).
 *   q[k]     wall fraction gamma in (0, 1]: the wall point is x_b = x_f + q e_d
 *            (the paper's x_b = x_f - gamma h e_i).
 *   uw       NULL (walls at rest) or 3*n_links wall velocities phi(x_b) (third
 *            component ignored in 2D), scaled per step by lbm_set_wall_factor.
 * Every fluid->solid pair must be listed exactly once; anything else is
 * LBM_EINVAL.  If the current scheme makes a link non-convex (Eq. 2.12) and
 * non-convex schemes were not allowed, LBM_ENONCONVEX.  Resets the populations
 * to rest. */
int lbm_set_geometry(lbm_ctx *ctx, const uint8_t *solid, int64_t n_links,
                     const int64_t *node, const int32_t *dir, const double *q,
                     const double *uw);

/* Family parameters (Sec. 2): l = c0 + c1*gamma + c2*gamma^2 (must be >= 0 for
 * every gamma in (0,1]), b in (0, 1] (Eq. 2.13).  Unless allow_nonconvex, every
 * link of the current geometry must satisfy max(0, 2g-1) <= l <= 2g (Eq. 2.12),
 * else LBM_ENONCONVEX and the previous scheme stays. */
int lbm_set_scheme(lbm_ctx *ctx, double c0, double c1, double c2, double b,
                   int allow_nonconvex);

/* Uniform body force g (lattice units, 3 components; g[2] ignored in 2D). */
int lbm_set_force(lbm_ctx *ctx, const double g[3]);

/* Two-node variant of the scheme (Sec. 2, Remark (2), Eq. 2.11): enable != 0 makes
 * every cut link whose node behind the boundary node, x_l = x_f + e_i, is fluid use
 * the exact f_ibar(x_f, t+1) = f'_ibar(x_l, t) in place of Eq. 2.9's f_ibar(x_f, t)
 * (within Eq. 2.13's b-combination); links with a solid x_l keep Eq. 2.10.  With
 * l = gamma this is the scheme of Yu, Mei & Shyy (2003) (Remark (4)).  Each step then
 * runs a small pass over those links before and after the sweep.  Stays on across
 * lbm_set_geometry.  lbm_adjoint and batches need it off (LBM_ESTATE).
 * Errors: LBM_ESTATE before lbm_set_geometry. */
int lbm_set_two_node(lbm_ctx *ctx, int enable);

/* Time-dependent wall velocity of the form phi(x_b, t) = a(t) phi_0(x_b) (Eq. 2.10's
 * phi evaluated at the time of the step, as in the paper's moving curved wall of
 * Sec. 3.2, whose field decays uniformly): from the current time t0 on, step t uses
 * every link's wall velocity (lbm_set_geometry / lbm_set_link_values) times
 * a(t) = a0 * r^(t - t0).  a0 = r = 1 (the default) is the constant wall.  The
 * adjoint (lbm_adjoint) follows the same factor step by step.  A batch uses each
 * member's factor for the member's time at the batch call, held for that call.
 * Errors: LBM_EINVAL for a non-finite a0 or r <= 0. */
int lbm_set_wall_factor(lbm_ctx *ctx, double a0, double r);

/* f = f^eq(rho, u) (Eq. 42) on fluid nodes.  rho: nodes doubles or NULL (rho0);
 * u: D*nodes doubles (D = 2 or 3, node-major) or NULL (rest).  Time resets to 0. */
int lbm_init_equilibrium(lbm_ctx *ctx, const double *rho, const double *u);

/* Full populations f_i(x, t) (not deviations), Q*nodes doubles, f[i*nodes + n].
 * set: values on solid nodes are ignored; time resets to 0.
 * get: NaN on solid nodes; valid after any number of steps. */
int lbm_set_populations(lbm_ctx *ctx, const double *f);
int lbm_get_populations(lbm_ctx *ctx, double *f);

/* Advance n >= 0 time steps (one fused collide-stream-boundary sweep each). */
int lbm_step(lbm_ctx *ctx, int n);
/* Number of steps taken since the last (re)initialisation. */
int64_t lbm_time(const lbm_ctx *ctx);

/* Density and reported velocity u = j/rho0 + g/2 (FP64) on fluid nodes, NaN on
 * solid nodes.  rho: nodes doubles or NULL; u: D*nodes doubles or NULL. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u);
/* Same into caller-owned device buffers (no synchronisation). */
int lbm_moments_device(lbm_ctx *ctx, double *rho_dev, double *u_dev);

/* Error norms over fluid nodes, reduced on the GPU in FP64 (Sec. 3.1, E_r):
 *   l2_rel  sqrt(sum |u_ref - u|^2) / sqrt(sum |u_ref|^2)   (u = LB velocity)
 *   linf    max |u_ref - u| (component-wise maximum)
 *   mass    sum of rho;  mom = sum of j = rho0 (u - g/2)
 *   residual sqrt(sum |u - u_prev|^2)/sqrt(sum |u|^2), u_prev = the velocity at
 *            the previous lbm_error_norms call (0 on the first call).
 * u_ref: D*nodes doubles (host), or NULL to skip l2_rel/linf (set to NaN).
 * Returns LBM_EDIVERGED (with the norms filled) if any density is non-finite. */
typedef struct {
  double l2_rel, linf, mass, mom[3], residual;
} lbm_norms;
int lbm_error_norms(lbm_ctx *ctx, const double *u_ref, lbm_norms *out);

/* Error norms without any allocation.  There is no counterpart in the paper: this
 * is a service entry point for callers that cannot allocate device memory when
 * they need the norms -- applications that give the whole device to their own
 * memory pool at start-up, services held to a fixed memory footprint, and tight
 * monitoring loops that cannot take the implicit synchronisation of
 * cudaMalloc/cudaFree.  It computes the same fluid-node sums as lbm_error_norms
 * but keeps its block partial sums in a static device array of the library
 * (80 KB, present on every GPU that loads the library until exit) and calls no
 * allocating routine.
 *   u_ref_dev  D*nodes doubles in device memory (node-major), or NULL to skip
 *              l2_rel and linf (written as NaN).
 *   out_dev    7 doubles in device memory, written on the context's stream:
 *              l2_rel, linf, mass, mom[0..2], number of non-finite densities.
 * No residual (it needs the per-context velocity history that lbm_error_norms
 * allocates).  Asynchronous: nothing is read back; synchronise the stream before
 * reading out_dev.
 * Limit: at most 33,554,432 nodes (e.g. 322^3); larger grids return LBM_EINVAL.
 * The first call on each device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  The looked-up address is kept for the life of the process: after a
 * cudaDeviceReset of that device it is stale, so do not call this entry point on
 * a device that was reset.  All calls share the array and it keeps the last call's
 * contents; calls that overlap on the GPU race on it, so issue them in order on one
 * stream. */
int lbm_error_norms_noalloc(lbm_ctx *ctx, const double *u_ref_dev, double *out_dev);

/* Limit on the sweep's wait for a tile's bulk copies, in polls of the tile's
 * barrier (each poll suspends for at most 1 ms); default 1000, about 1 s, far
 * beyond any legitimate copy latency.  There is no counterpart in the paper: it
 * is the failure-detection bound of the library's pipeline.  A warp whose wait
 * runs out sets the context's status (read as LBM_ETIMEOUT by the next
 * lbm_moments or lbm_error_norms), waits with the default limit for the copies it
 * still has in flight and leaves the step unfinished; a new initial state
 * (lbm_init_equilibrium or lbm_set_populations) clears the status.  polls = 0
 * makes every sweep give up at its first wait, which exercises that path without
 * any fault.  polls < 0 is LBM_EINVAL.  Batches use the default limit. */
int lbm_set_wait_limit(lbm_ctx *ctx, int polls);

/* Replace the relaxation rates (no reset of the populations). */
int lbm_set_relaxation(lbm_ctx *ctx, const double *s);

/* Replace the wall fractions and/or wall velocities of the existing cut links
 * (same list, same order as given to lbm_set_geometry; NULL keeps the current
 * values), with the checks of lbm_set_geometry and lbm_set_scheme.  The
 * populations are not reset. */
int lbm_set_link_values(lbm_ctx *ctx, const double *q, const double *uw);

/* Discrete adjoint of n_steps time steps from the current state (reverse mode of
 * exactly what lbm_step computes), for the loss
 *   J = sum over fluid nodes n with mask[n] != 0 of |u(x_n, T) - u_target(x_n)|^2,
 * u the reported velocity after the n_steps (T = current time + n_steps).
 * The forward run keeps a raw checkpoint every checkpoint_every steps (0 = about
 * sqrt(n_steps)); the backward pass recomputes one segment at a time from its
 * checkpoint and runs the adjoint sweep through it.  On return the context is in
 * the state after the forward run (as if lbm_step(n_steps) had been called).
 *   mask      nodes bytes (host); u_target D*nodes doubles (host, node-major).
 *   loss      J (may be NULL).
 *   grad_s    Q doubles: dJ/ds_k (0 for the conserved rows), or NULL.
 *   grad_q    n_links doubles: dJ/dq per link in the order given to
 *             lbm_set_geometry, or NULL.
 *   grad_uw   3*n_links doubles: dJ/dphi per link, or NULL.
 * The adjoint computes in double for LBM_F64 and in float otherwise; gradients
 * are accumulated in double.  Memory: about (n_steps/checkpoint_every +
 * checkpoint_every + 3) population arrays, kept in the context after a successful
 * call and reused (grown when needed) by later calls; lbm_destroy releases it. */
int lbm_adjoint(lbm_ctx *ctx, int n_steps, int checkpoint_every, const uint8_t *mask,
                const double *u_target, double *loss, double *grad_s, double *grad_q,
                double *grad_uw);

/* lbm_adjoint in two halves, for a reverse-mode framework whose forward and
 * backward calls are separate (lbm_adjoint is exactly the two in sequence).
 * lbm_adjoint_forward runs the n_steps with checkpoints, keeps the tape (the
 * checkpoints, the last segment's states, mask and u_target) in the context and
 * returns J; its cost is that of lbm_step(n_steps) plus the checkpoint copies.
 * lbm_adjoint_backward recomputes and runs the adjoint sweep from that tape and
 * returns the gradients; the context ends in the forward run's end state, and the
 * tape stays valid, so the backward pass may be repeated.  Any call that changes
 * the populations or the arguments of the step in between (lbm_step,
 * lbm_init_equilibrium, lbm_set_populations, lbm_set_geometry, lbm_set_relaxation,
 * lbm_set_link_values, lbm_set_scheme, lbm_set_force, lbm_set_wall_factor, a batch
 * step) discards the tape: lbm_adjoint_backward then returns LBM_ESTATE.  One tape
 * per context; a new forward pass replaces it.  Arguments as for lbm_adjoint. */
int lbm_adjoint_forward(lbm_ctx *ctx, int n_steps, int checkpoint_every, const uint8_t *mask,
                        const double *u_target, double *loss);
int lbm_adjoint_backward(lbm_ctx *ctx, double *grad_s, double *grad_q, double *grad_uw);

/* Batches (ensembles of independent problems).  A batch advances several contexts
 * -- same lattice, precision and device, any sizes, geometries and parameters --
 * by ONE persistent sweep launch per time step that walks the tiles of all of them,
 * replayed from a CUDA graph holding an even and an odd step.  Each context keeps
 * its own state; stepping a batch is equivalent (bit for bit) to stepping every
 * context alone.  Contexts are borrowed: they must outlive the batch, and they must
 * be at the same time parity when the batch steps.  Changes to a member context
 * (geometry, scheme, force) are picked up at the next batch call.
 * lbm_batch_set_config: order of tiles in the launch (0 context after context,
 * 1 round-robin over contexts, 2 largest context first), resident blocks per SM
 * (0 = as many as fit) and split: 1 (the default) gives every kernel class of
 * members -- rows starting on 16-byte boundaries or not, skewed x-wrap or not --
 * its own launch of the sweep specialised for it (aligned windows, no skew
 * handling), all inside the same graph; 0 runs every member through the general
 * sweep (unaligned windows, skew), one launch per step.  tile_w: nodes per warp
 * tile, 64 (the default, as for a single context) or 32 (every 64-node tile cut
 * in halves, halves without fluid dropped: fewer idle lanes on small or thin
 * members, more pipeline work per node).  The results do not depend on order,
 * blocks, split or tile_w, bit for bit.  Grids whose slots need 64-bit indices
 * always take the general sweep in 64-node tiles.  lbm_batch_tune times every
 * (tile_w, split, order, blocks) combination over trial_steps steps, keeps the
 * fastest and restores the contexts' state, so tuning does not advance the
 * simulations; any output pointer may be NULL.  lbm_batch_query also reports the
 * kernel launches one step takes and the tile width in use.  LBM_EINVAL for a
 * value out of range. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_batch **out, int n, lbm_ctx *const *ctxs);
int lbm_batch_destroy(lbm_batch *batch);
int lbm_batch_set_stream(lbm_batch *batch, void *cuda_stream);
int lbm_batch_set_config(lbm_batch *batch, int order, int blocks_per_sm, int split, int tile_w);
int lbm_batch_tune(lbm_batch *batch, int trial_steps, int *order, int *blocks_per_sm, int *split,
                   int *tile_w);
int lbm_batch_step(lbm_batch *batch, int n);
int lbm_batch_query(const lbm_batch *batch, int *n_contexts, int64_t *tiles, int *order,
                    int *blocks_per_sm, int *launches_per_step, int *tile_w);
const char *lbm_batch_last_error(const lbm_batch *batch);

/* The current device's FP64 fused multiply-add rate in GFLOP/s (an FMA counted as
 * two operations), measured with a plain timed FMA loop (8 independent chains per
 * thread, every SM full).  There is no counterpart in the paper: it is the
 * denominator against which the FP64 sweep, bound by the FP64 pipe rather than by
 * HBM on this GPU, is reported.  Runs on the legacy stream and synchronises it;
 * changes no device setting.  LBM_EINVAL for a NULL pointer, LBM_ECUDA if a CUDA
 * call fails. */
int lbm_probe_fp64_rate(double *gflops);

/* Sizes: lattice Q and D, node counts, link count. */
int lbm_query(const lbm_ctx *ctx, int *Q, int *D, int64_t *nodes, int64_t *fluid_nodes,
              int64_t *links);

/* Message of the last failing call on ctx (or of the last failed lbm_create when
 * ctx is NULL).  Never NULL. */
const char *lbm_last_error(const lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
