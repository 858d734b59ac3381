"""D3Q15, the paper's own 3D lattice (Appendix: velocities, weights and M as printed,
S of Sec. 3), through the C-ABI against the FP64 oracle: element-wise parity of
the fused sweep and of the discrete adjoint, reduced-precision bounds, batches, and
second order on the paper's Hagen-Poiseuille pipe (Sec. 3.3, axis along x)."""

import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import lattices as OL
from oracle import lbm as O
from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import check_close, deviation, gpu_sim, oracle_sim, require_gpu

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
LAT = "D3Q15"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _sphere_ragged(seed=5):
    n = 13
    w = W.sphere_3d(n, 3.3, (6.2, 4.9, 4.4), s_nu=1.1, force=(1e-5, 2e-6, -3e-6), lattice=LAT)
    solid = np.asarray(w["solid"]).reshape(n, n, n).copy()
    solid[:, 11:, :] = True
    solid[9:, :, :] = True
    w["solid"] = solid.ravel()
    node, d = W.cut_links(LAT, w["shape"], (0, 0), w["solid"])
    rng = np.random.default_rng(seed)
    w["links"] = dict(node=node, d=d, q=rng.uniform(0.05, 1.0, len(node)),
                      uw=0.01 * rng.standard_normal((len(node), 3)))
    return w


def _u_oracle(o):
    _, u = o.moments()
    return u


def test_relaxation_vector_is_the_printed_one():
    s = W.relaxation_rates(LAT, 1.37)
    assert s.tolist() == [1, 1.8, 1.2, 1, 0.5, 1, 0.5, 1, 0.5, 1.37, 1.37, 1.37, 1.37, 1.37, 1.5]
    assert np.array_equal(W.DIRECTIONS[LAT], OL.D3Q15.e)


@pytest.mark.parametrize("steps", [1, 2, 17])
@pytest.mark.parametrize("scheme", [(0, 1, 0, 1.0), (0, 1, 1, 0.8)])
def test_sphere_ragged_box(steps, scheme):
    """A sphere in a ragged periodic box (walls on the wrap), random state and wall
    velocities, body force: every population against the oracle."""
    w = _sphere_ragged()
    rho, u = W.random_state(w["shape"], LAT, 1.0, 0.01, seed=6)
    o = oracle_sim(w, scheme=scheme)
    o.init_equilibrium(rho, u)
    o.step(steps)
    g = gpu_sim(w, "f64", scheme=scheme)
    g.init_equilibrium(rho, u)
    g.step(steps)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), OL.D3Q15), deviation(o.f, OL.D3Q15), TOL64, fl)


@pytest.mark.parametrize("L", [16, 32])
def test_tilted_pipe_skewed_wrap(L):
    """The tilted pipe with the skewed x-wrap, random perturbation of the analytic
    start: L = 16 (one tile holds both x-edges of a row) and L = 32."""
    w = W.tilted_pipe_3d(L, lattice=LAT)
    rho, u = W.random_state(w["shape"], LAT, 1.0, 0.002, seed=9)
    u = u + np.nan_to_num(w["u_exact"])
    o = oracle_sim(w)
    o.init_equilibrium(rho, u)
    o.step(31)
    g = gpu_sim(w, "f64")
    g.init_equilibrium(rho, u)
    g.step(31)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), OL.D3Q15), deviation(o.f, OL.D3Q15), TOL64, fl)


def test_ragged_row_length_unaligned_windows():
    """nx = 37 (rows not on 16-byte boundaries: the unaligned-window path)."""
    shape = (37, 12, 10)
    N = shape[0] * shape[1] * shape[2]
    y = (np.arange(N) // shape[0]) % shape[1]
    solid = (y == 0) | (y == 11)
    node, d = W.cut_links(LAT, shape, (0, 0), solid)
    rng = np.random.default_rng(3)
    w = dict(lattice=LAT, shape=shape, skew=(0, 0), solid=solid,
             links=dict(node=node, d=d, q=rng.uniform(0.1, 1.0, len(node)),
                        uw=0.01 * rng.standard_normal((len(node), 3))),
             S=W.relaxation_rates(LAT, 1.3), rho0=1.0, force=(2e-6, 0.0, 1e-6))
    rho, u = W.random_state(shape, LAT, 1.0, 0.01, seed=4)
    o = oracle_sim(w)
    o.init_equilibrium(rho, u)
    o.step(9)
    g = gpu_sim(w, "f64")
    g.init_equilibrium(rho, u)
    g.step(9)
    check_close(deviation(g.get_populations(), OL.D3Q15), deviation(o.f, OL.D3Q15), TOL64, ~solid)


@pytest.mark.parametrize("prec,tol", [("f32", 2e-6), ("bf16", 5e-2), ("f16", 1e-2)])
def test_reduced_precision_pipe(prec, tol):
    w = W.tilted_pipe_3d(32, lattice=LAT)
    u0 = np.nan_to_num(w["u_exact"])
    o = oracle_sim(w)
    o.init_equilibrium(None, u0)
    o.step(200)
    g = gpu_sim(w, prec)
    g.init_equilibrium(None, u0)
    g.step(200)
    fl = ~w["solid"]
    _, ug = g.moments()
    check_close(ug[fl], _u_oracle(o)[fl], tol, None, "D3Q15 %s pipe u" % prec)


def test_batch_equals_individual_steps():
    torch = require_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    ws = [W.tilted_pipe_3d(16, lattice=LAT), _sphere_ragged(7)]
    solo, grouped = [], []
    for k, w in enumerate(ws):
        for lst in (solo, grouped):
            s = gpu_sim(w, "f32")
            rho, u = W.random_state(w["shape"], LAT, 1.0, 0.005, seed=20 + k)
            s.init_equilibrium(rho, u)
            s.set_stream(stream)
            lst.append(s)
    batch = B.Batch(grouped)
    batch.set_stream(stream)
    for s in solo:
        s.step(5)
    batch.step(5)
    for a, b, w in zip(solo, grouped, ws):
        fl = ~w["solid"]
        assert np.array_equal(a.get_populations()[:, fl], b.get_populations()[:, fl])
    batch.close()


@pytest.mark.parametrize("scheme", [(0, 1, 0, 1.0), (0, 1, 1, 0.7)])
def test_fp64_adjoint_equals_oracle_adjoint(scheme):
    w = W.sphere_3d(6, 1.7, (2.6, 3.1, 2.4), s_nu=1.1, force=(1e-5, 0.0, 2e-5), lattice=LAT)
    w["links"] = W.random_links_uw(w["links"], 0.01, seed=3)
    N = 6 ** 3
    rng = np.random.default_rng(7)
    rho, u = W.random_state(w["shape"], LAT, 1.0, 0.01, seed=8)
    mask = rng.random(N) < 0.5
    ut = 0.01 * rng.standard_normal((N, 3))
    o = O.Simulation(OL.D3Q15, w["shape"], w["S"], 1.0, w["solid"], w["links"], scheme=scheme,
                     force=w["force"])
    o.init_equilibrium(rho, u)
    J0, gs0, gq0, gp0 = OA.adjoint(o, 5, mask, ut)
    g = gpu_sim(w, "f64", scheme=scheme)
    g.init_equilibrium(rho, u)
    J, gs, gq, gp = g.adjoint(5, mask, ut, checkpoint_every=2)
    assert abs(J - J0) <= 1e-12 * abs(J0)
    # every gradient entry within 1e-10 of the largest gradient of its own kind
    check_close(gs, gs0, 1e-10, None, "D3Q15 dJ/ds")
    check_close(gq, gq0, 1e-10, None, "D3Q15 dJ/dq")
    check_close(gp, gp0, 1e-10, None, "D3Q15 dJ/dphi")


def test_hagen_poiseuille_second_order():
    """The paper's Sec. 3.3 setup: a pipe along x (radius 0.4 L), body force, FP64
    to a steady state; the error against the parabola falls at second order."""
    sizes = [16, 32]
    errs = []
    for L in sizes:
        w = W.tilted_pipe_3d(L, axis_dir=(1, 0, 0), lattice=LAT)
        ue = np.nan_to_num(w["u_exact"])
        g = gpu_sim(w, "f64")
        g.init_equilibrium(None, ue)
        g.error_norms(ue)
        res, steps = 1.0, 0
        while res > 1e-10:
            assert steps < 200000
            g.step(200)
            steps += 200
            res = g.error_norms(ue)["residual"]
        errs.append(g.error_norms(ue)["l2_rel"])
    order = np.log(errs[0] / errs[1]) / np.log(2)
    print("D3Q15 pipe E_r", errs, "order", order)
    assert order >= 1.8, errs
