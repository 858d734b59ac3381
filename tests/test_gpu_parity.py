"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the same
seeded inputs, element by element.

Tolerances.  FP64 storage: 1e-12 relative (norm-wise over the compared entries)
on velocities, and on population deviations g = f - w rho0 for runs of up to a
few hundred steps.  Over thousands of steps the oracle's own rounding sets the
floor: it stores full f (about w rho0), so each boundary update carries a
systematic error of order eps*|f| that accumulates linearly in the deviations
(a deviation-form evaluation of the same equations differs from the oracle by
4.2e-11 deviation-relative after 3000 steps of the 64^2 Couette problem); long
runs therefore compare populations relative to |f|, at 1e-12.
Reduced-precision storage keeps deviations, computes in FP32 and is held to
stated bounds on u measured against the oracle: FP32 2e-6, BF16 5e-2, FP16 1e-2
after 3000 steps of the 64^2 Couette problem (measured 6.0e-8, 2.8e-2, 4.4e-3).
"""

import numpy as np
import pytest

from oracle import lattices as OL
from oracle import lbm as O
from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import check_close, deviation, gpu_sim, oracle_sim, patch_reference, require_gpu

pytestmark = pytest.mark.gpu

RULES = [(0, 1, 0), (0, 1.5, 0), (0, 2, 0), (0, 0, 1), (0, 1, 1)]
TOL64 = 1e-12
TOL_U = {"f32": 2e-6, "bf16": 5e-2, "f16": 1e-2}
# FP32 deviations over a few steps: a step rounds each deviation a few times at
# 2^-24 relative to the largest deviation in play
TOL32_STEPS = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _u_oracle(sim):
    _, u = sim.moments()
    return u[:, : sim.lat.D]


def test_rest_state_stays_exact_all_precisions():
    w = W.couette_config(48)
    w = dict(w)
    w["links"] = dict(w["links"], uw=np.zeros_like(w["links"]["uw"]))
    for prec in ("f64", "f32", "bf16", "f16"):
        g = gpu_sim(w, prec, scheme=(0, 1, 1, 0.7))
        g.init_equilibrium()
        g.step(7)
        f = g.get_populations()
        fl = ~w["solid"]
        assert np.array_equal(f[:, fl], np.repeat(OL.D2Q9.w[:, None], fl.sum(), 1)), prec


def test_couette_64_f64_3000_steps():
    """The 64^2 circular Couette problem, rest start, 3000 steps, default family
    parameters (l = gamma, b = 1): GPU FP64 equals the oracle to 1e-12."""
    w = W.couette_config(64)
    o = oracle_sim(w)
    o.init_equilibrium()
    o.step(3000)
    g = gpu_sim(w, "f64")
    g.init_equilibrium()
    g.step(3000)
    fl = ~w["solid"]
    _, ug = g.moments()
    check_close(ug[fl], _u_oracle(o)[fl], TOL64, None)
    fg = g.get_populations()
    check_close(fg, o.f, TOL64, fl)
    # the deviations agree to the oracle's own accumulated rounding (see module doc)
    check_close(deviation(fg, OL.D2Q9), deviation(o.f, OL.D2Q9), 1e-10, fl)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("b", [1.0, 0.55])
def test_d2q9_family_random_walls(rule, b):
    """Every l-rule of Sec. 3 and a b < 1 (Eq. 2.13), random wall velocities on every
    link, a ragged 37 x 29 grid, an odd number of steps (AA odd layout read back)."""
    w = W.couette_2d(37, (18.2, 14.1), 4.3, 13.1, 0.0)
    w.update(S=W.relaxation_rates("D2Q9", 1.3), rho0=1.0, force=(2e-6, -1e-6, 0.0))
    w["links"] = W.random_links_uw(w["links"], 0.01, seed=11)
    w["shape"] = (37, 37, 1)
    rho, u = W.random_state(w["shape"], "D2Q9", 1.0, 0.01, seed=12)
    sc = tuple(rule) + (b,)
    o = oracle_sim(w, scheme=sc)
    o.init_equilibrium(rho, u)
    o.step(41)
    g = gpu_sim(w, "f64", scheme=sc)
    g.init_equilibrium(rho, u)
    g.step(41)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), OL.D2Q9), deviation(o.f, OL.D2Q9), TOL64, fl)
    _, ug = g.moments()
    check_close(ug[fl], _u_oracle(o)[fl], TOL64, None)


@pytest.mark.parametrize("steps", [1, 2, 17])
def test_d3q19_sphere_ragged_box(steps):
    """D3Q19, a sphere in a ragged 13 x 11 x 9 periodic box (walls reach the wrap),
    random state and wall velocities, l = gamma^2 + gamma, b = 0.8, body force."""
    w = W.sphere_3d(13, 3.3, (6.2, 4.9, 4.4), s_nu=1.1, force=(1e-5, 2e-6, -3e-6))
    w["shape"] = (13, 13, 13)
    # carve a ragged box: make the last rows/planes solid so nx, ny, nz differ in effect
    solid = np.asarray(w["solid"]).reshape(13, 13, 13).copy()
    solid[:, 11:, :] = True
    solid[9:, :, :] = True
    w["solid"] = solid.ravel()
    node, d = W.cut_links("D3Q19", w["shape"], (0, 0), w["solid"])
    rng = np.random.default_rng(5)
    w["links"] = dict(node=node, d=d, q=rng.uniform(0.05, 1.0, len(node)),
                      uw=0.01 * rng.standard_normal((len(node), 3)))
    rho, u = W.random_state(w["shape"], "D3Q19", 1.0, 0.01, seed=6)
    sc = (0, 1, 1, 0.8)
    o = oracle_sim(w, scheme=sc)
    o.init_equilibrium(rho, u)
    o.step(steps)
    g = gpu_sim(w, "f64", scheme=sc)
    g.init_equilibrium(rho, u)
    g.step(steps)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), OL.D3Q19), deviation(o.f, OL.D3Q19), TOL64, fl)


def test_d3q19_tilted_pipe_skewed_wrap():
    """The tilted periodic pipe at L = 32 (skewed x-wrap), analytic start plus noise,
    60 steps: FP64 parity on every population."""
    w = W.tilted_pipe_3d(32)
    rho, u = W.random_state(w["shape"], "D3Q19", 1.0, 0.002, seed=9)
    u = u + np.nan_to_num(w["u_exact"])
    o = oracle_sim(w)
    o.init_equilibrium(rho, u)
    o.step(60)
    g = gpu_sim(w, "f64")
    g.init_equilibrium(rho, u)
    g.step(60)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), OL.D3Q19), deviation(o.f, OL.D3Q19), TOL64, fl)


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
def test_reduced_precision_bounds_couette(prec):
    """Deviation storage in FP32/BF16/FP16, FP32 arithmetic: velocity error against
    the FP64 oracle after 3000 steps of the 64^2 Couette problem within the stated
    bound."""
    w = W.couette_config(64)
    o = oracle_sim(w)
    o.init_equilibrium()
    o.step(3000)
    g = gpu_sim(w, prec)
    g.init_equilibrium()
    g.step(3000)
    fl = ~w["solid"]
    _, ug = g.moments()
    check_close(ug[fl], _u_oracle(o)[fl], TOL_U[prec], None, "%s couette u" % prec)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_reduced_precision_d3q19_pipe(prec):
    w = W.tilted_pipe_3d(32)
    u0 = np.nan_to_num(w["u_exact"])
    o = oracle_sim(w)
    o.init_equilibrium(None, u0)
    o.step(200)
    g = gpu_sim(w, prec)
    g.init_equilibrium(None, u0)
    g.step(200)
    fl = ~w["solid"]
    _, ug = g.moments()
    check_close(ug[fl], _u_oracle(o)[fl], TOL_U[prec], None, "%s pipe u" % prec)


def test_populations_round_trip_and_parity_layouts():
    """set -> get is the identity (FP64), also after stepping an odd number of
    steps and back through the other layout."""
    w = W.tilted_pipe_3d(16)
    rng = np.random.default_rng(3)
    f = OL.D3Q19.w[:, None] * (1 + 0.01 * rng.standard_normal((19, 16 ** 3)))
    g = gpu_sim(w, "f64")
    g.set_populations(f)
    fl = ~w["solid"]
    back = g.get_populations()
    assert np.array_equal(back[:, fl], f[:, fl])
    assert np.isnan(back[:, ~fl]).all()
    o = oracle_sim(w)
    ff = f.copy()
    ff[:, ~fl] = np.nan
    o.f = ff
    o.step(3)
    g.step(3)
    check_close(deviation(g.get_populations(), OL.D3Q19), deviation(o.f, OL.D3Q19), TOL64, fl)


def test_error_norms_match_host_formula():
    w = W.couette_config(64)
    g = gpu_sim(w, "f64")
    g.init_equilibrium()
    g.step(500)
    fl = ~w["solid"]
    rho, u = g.moments()
    ue = w["u_exact"][:, :2]
    nrm = g.error_norms(np.nan_to_num(ue))
    want = O.relative_l2_error(ue, u, fl)
    assert abs(nrm["l2_rel"] - want) < 1e-12 * want
    assert abs(nrm["mass"] - rho[fl].sum()) < 1e-12 * rho[fl].sum()
    assert abs(nrm["linf"] - np.abs(ue[fl] - u[fl]).max()) < 1e-15
    # residual: second call sees the previous velocity
    g.step(10)
    n2 = g.error_norms(None)
    _, u2 = g.moments()
    want_res = np.sqrt(((u2[fl] - u[fl]) ** 2).sum() / (u2[fl] ** 2).sum())
    assert abs(n2["residual"] - want_res) < 1e-10 * want_res


def test_full_size_pipe_sampled_nodes():
    """The L = 256 tilted pipe (16.8M nodes), the launch configuration the bench
    times, FP64 and FP32 storage: 2 steps from a perturbed analytic start; 64 sampled
    nodes (boundary, interior and wrap-edge nodes) against the oracle's patch
    evaluation."""
    L = 256
    w = W.tilted_pipe_3d(L)
    lat = OL.D3Q19
    rng = np.random.default_rng(21)
    N = L ** 3
    rho = 1.0 + 0.001 * rng.standard_normal(N)
    u = np.nan_to_num(w["u_exact"]) + 0.001 * rng.standard_normal((N, 3))
    fl = np.nonzero(~w["solid"])[0]
    bnd = np.unique(w["links"]["node"])
    x = fl % L
    edge = fl[(x == 0) | (x == L - 1)]
    centres = np.concatenate([rng.choice(bnd, 24, replace=False), rng.choice(fl, 24, replace=False),
                              rng.choice(edge, 16, replace=False)])
    k = 2
    f0_fn = lambda idx: O.equilibrium(lat, rho[idx], u[idx].T, 1.0)
    want = patch_reference(w, f0_fn, centres, k, (0, 1, 0, 1.0))
    for prec, tol in (("f64", TOL64), ("f32", TOL32_STEPS)):
        g = gpu_sim(w, prec)
        g.init_equilibrium(rho, u)
        g.step(k)
        f = g.get_populations()[:, centres]
        check_close(deviation(f, lat), deviation(want, lat), tol, None, "%s L=256 samples" % prec)
        del g


@pytest.mark.parametrize("kind", ["bgk", "trt"])
def test_other_collision_operators_through_the_same_sweep(kind):
    """Remark (1) after Eq. 2.10: the boundary construction does not depend on the
    collision.  BGK and TRT, written as MRT relaxation vectors, run through the same
    sweep and boundary against the oracle (D2Q9 Couette with random walls, D3Q19
    sphere box)."""
    cases = []
    w2 = W.couette_config(64)
    w2["links"] = W.random_links_uw(w2["links"], 0.01, seed=8)
    cases.append((w2, OL.D2Q9))
    w3 = W.sphere_3d(12, 3.1, (5.7, 6.2, 5.4), s_nu=1.1, force=(1e-5, 0.0, 2e-6))
    w3["links"] = W.random_links_uw(w3["links"], 0.01, seed=9)
    cases.append((w3, OL.D3Q19))
    for w, lat in cases:
        w = dict(w)
        w["S"] = (W.relaxation_rates_bgk(lat.name, 1.25) if kind == "bgk"
                  else W.relaxation_rates_trt(lat.name, 1.25))
        rho, u = W.random_state(w["shape"], lat.name, 1.0, 0.01, seed=10)
        o = oracle_sim(w, scheme=(0, 1, 1, 0.9))
        o.init_equilibrium(rho, u)
        o.step(23)
        g = gpu_sim(w, "f64", scheme=(0, 1, 1, 0.9))
        g.init_equilibrium(rho, u)
        g.step(23)
        fl = ~w["solid"]
        check_close(deviation(g.get_populations(), lat), deviation(o.f, lat), TOL64, fl)


@pytest.mark.parametrize("lattice,shape,skew,prec", [
    ("D2Q9", (1, 9, 1), (0, 0), "f64"),     # one column: every node on both x-edges
    ("D2Q9", (2, 7, 1), (0, 0), "f64"),
    ("D2Q9", (3, 1, 1), (0, 0), "f64"),     # one row, no walls, no cut links
    ("D3Q19", (1, 6, 5), (2, 1), "f64"),    # one column with a skewed x-wrap
    ("D3Q19", (2, 5, 4), (0, 0), "f32"),
    ("D3Q15", (1, 4, 4), (1, 3), "f64"),
    ("D3Q19", (65, 4, 3), (0, 0), "f64"),   # a full tile plus a one-node tile per row
    # FP64 sweeps run 32-node half tiles: the x = nx-1 edge in the second half, in the
    # only half (both edges in one tile), and a ragged one-node half, with skew
    ("D3Q19", (40, 5, 4), (1, 2), "f64"),
    ("D3Q19", (24, 4, 5), (2, 1), "f64"),
    ("D2Q9", (33, 6, 1), (0, 0), "f64"),
])
def test_thin_and_degenerate_grids(lattice, shape, skew, prec):
    """Grids one or two nodes thick, a single row, and a ragged last tile: walls on the
    first and last rows when there are at least four, random wall fractions and wall
    velocities, random state, seven steps (both parities) against the oracle."""
    nx, ny, nz = shape
    N = nx * ny * nz
    y = (np.arange(N) // nx) % ny
    solid = (y == 0) | (y == ny - 1) if ny >= 4 else np.zeros(N, bool)
    node, d = W.cut_links(lattice, shape, skew, solid)
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    w = dict(lattice=lattice, shape=shape, skew=skew, solid=solid,
             links=dict(node=node, d=d, q=rng.uniform(0.1, 1.0, len(node)),
                        uw=0.01 * rng.standard_normal((len(node), 3))),
             S=W.relaxation_rates(lattice, 1.2), rho0=1.0, force=(1e-5, -2e-6, 3e-6))
    rho, u = W.random_state(shape, lattice, 1.0, 0.01, seed=3)
    lat = OL.BY_NAME[lattice]
    o = oracle_sim(w, scheme=(0, 1, 1, 0.9))
    o.init_equilibrium(rho, u)
    o.step(7)
    g = gpu_sim(w, prec, scheme=(0, 1, 1, 0.9))
    g.init_equilibrium(rho, u)
    g.step(7)
    fl = ~solid
    check_close(deviation(g.get_populations(), lat), deviation(o.f, lat),
                TOL64 if prec == "f64" else TOL32_STEPS, fl, "%s %s %s" % (lattice, shape, prec))


def test_full_size_couette_2048_sampled_nodes():
    """The refinement study's largest grid (2048^2, D2Q9), FP64 and FP32: 3 steps from
    a perturbed analytic start; 48 sampled nodes (both walls, interior) against the
    oracle's patch evaluation."""
    n = 2048
    w = W.couette_config(n)
    lat = OL.D2Q9
    rng = np.random.default_rng(22)
    N = n * n
    rho = 1.0 + 0.001 * rng.standard_normal(N)
    u = np.nan_to_num(w["u_exact"]) + 0.0005 * rng.standard_normal((N, 3))
    u[:, 2] = 0.0
    fl = np.nonzero(~w["solid"])[0]
    bnd = np.unique(w["links"]["node"])
    centres = np.concatenate([rng.choice(bnd, 32, replace=False), rng.choice(fl, 16, replace=False)])
    k = 3
    f0_fn = lambda idx: O.equilibrium(lat, rho[idx], u[idx].T, 1.0)
    want = patch_reference(w, f0_fn, centres, k, (0, 1, 0, 1.0))
    for prec, tol in (("f64", TOL64), ("f32", TOL32_STEPS)):
        g = gpu_sim(w, prec)
        g.init_equilibrium(rho, u[:, :2])
        g.step(k)
        check_close(deviation(g.get_populations()[:, centres], lat), deviation(want, lat), tol, None,
                    "%s 2048^2 samples" % prec)
        del g


def test_full_size_d3q15_pipe_sampled_nodes():
    """The bench's D3Q15 section size (L = 256 pipe), FP32, 2 steps, sampled nodes."""
    L = 256
    w = W.tilted_pipe_3d(L, lattice="D3Q15")
    lat = OL.D3Q15
    rng = np.random.default_rng(23)
    N = L ** 3
    rho = 1.0 + 0.001 * rng.standard_normal(N)
    u = np.nan_to_num(w["u_exact"]) + 0.001 * rng.standard_normal((N, 3))
    fl = np.nonzero(~w["solid"])[0]
    bnd = np.unique(w["links"]["node"])
    x = fl % L
    edge = fl[(x == 0) | (x == L - 1)]
    centres = np.concatenate([rng.choice(bnd, 16, replace=False), rng.choice(fl, 8, replace=False),
                              rng.choice(edge, 8, replace=False)])
    f0_fn = lambda idx: O.equilibrium(lat, rho[idx], u[idx].T, 1.0)
    want = patch_reference(w, f0_fn, centres, 2, (0, 1, 0, 1.0))
    g = gpu_sim(w, "f32")
    g.init_equilibrium(rho, u)
    g.step(2)
    check_close(deviation(g.get_populations()[:, centres], lat), deviation(want, lat), TOL32_STEPS,
                None, "D3Q15 f32 L=256 samples")


def test_64bit_slot_indices_periodic_box():
    """A grid whose population slots need 64-bit element indices (Q * S >= 2^31: a
    484^3 D3Q19 periodic box, 113M nodes, FP32): the sweep's long-index
    instantiations (even and odd steps) against the oracle on sampled nodes.  A
    density perturbation makes the field non-uniform; after 2 steps rho and u of 24
    sampled nodes are compared with the oracle's patch evaluation."""
    torch = require_gpu()
    n = 484
    N = n ** 3
    assert 19 * N >= 2 ** 31
    lat = OL.D3Q19
    x = np.arange(N) % n
    y = (np.arange(N) // n) % n
    z = np.arange(N) // (n * n)
    rho = 1.0 + 1e-3 * (np.sin(2 * np.pi * x / 37.0) + np.cos(2 * np.pi * y / 53.0) * np.sin(2 * np.pi * z / 29.0))
    del x, y, z
    S = W.relaxation_rates("D3Q19", 1.3)
    g = B.Lbm("D3Q19", (n, n, n), S, "f32")
    g.set_force((1e-5, -2e-6, 3e-6))
    g.init_equilibrium(rho, None)
    g.step(2)
    rho_g, u_g = g.moments()
    g.close()
    w = dict(lattice="D3Q19", shape=(n, n, n), skew=(0, 0), solid=np.zeros(N, bool),
             links=dict(node=np.zeros(0, np.int64), d=np.zeros(0, np.int64), q=np.zeros(0),
                        uw=np.zeros((0, 3))),
             S=S, rho0=1.0, force=(1e-5, -2e-6, 3e-6))
    rng = np.random.default_rng(24)
    centres = rng.choice(N, 24, replace=False)
    f0_fn = lambda idx: O.equilibrium(lat, rho[idx], np.zeros((3, len(idx))), 1.0)
    want = patch_reference(w, f0_fn, centres, 2, (0, 1, 0, 1.0))
    e = lat.e.T.astype(float)
    rho_w = want.sum(axis=0)
    u_w = (e @ want).T / 1.0 + 0.5 * np.array([1e-5, -2e-6, 3e-6])
    check_close(rho_g[centres] - 1.0, rho_w - 1.0, TOL32_STEPS, None, "64-bit index rho - 1")
    check_close(u_g[centres], u_w, 1e-5, None, "64-bit index u")
