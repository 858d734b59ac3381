"""GPU discrete adjoint (lbm_adjoint) against the oracle's FP64 discrete adjoint and
against central finite differences of the GPU forward run.

Tolerances: FP64 GPU vs oracle adjoint 1e-10 relative to the largest gradient
(different summation order over nodes and steps); FP64 adjoint vs central
differences with h = 1e-4 (the bound the design targets), 1e-4 relative to the
gradient scale; FP32 adjoint vs FP64 adjoint 1e-3 (measured and stated in the
design notes)."""

import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import lattices as OL
from oracle import lbm as O
from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import gpu_sim, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case(kind):
    if kind == "couette":
        w = W.couette_2d(14, (7.2, 6.9), 2.1, 6.1, 0.01)
        w["links"] = W.random_links_uw(w["links"], 0.01, seed=1)
        rng = np.random.default_rng(2)
        w["links"]["q"] = rng.uniform(0.1, 1.0, len(w["links"]["q"]))
        w.update(S=W.relaxation_rates("D2Q9", 1.3), rho0=1.0, force=(2e-5, -1e-5, 0.0))
        return w
    if kind == "sphere":
        w = W.sphere_3d(6, 1.7, (2.6, 3.1, 2.4), s_nu=1.1, force=(1e-5, 0.0, 2e-5))
        w["links"] = W.random_links_uw(w["links"], 0.01, seed=3)
        return w
    if kind == "pipe":
        w = W.tilted_pipe_3d(16)
        w["links"] = W.random_links_uw(w["links"], 0.005, seed=4)
        return w
    raise ValueError(kind)


def _inputs(w, seed):
    N = w["shape"][0] * w["shape"][1] * w["shape"][2]
    D = 2 if w["lattice"] == "D2Q9" else 3
    rng = np.random.default_rng(seed)
    rho, u = W.random_state(w["shape"], w["lattice"], 1.0, 0.01, seed=seed + 1)
    mask = rng.random(N) < 0.5
    ut = 0.01 * rng.standard_normal((N, D))
    return rho, u, mask, ut


@pytest.mark.parametrize("kind,steps,ckpt", [("couette", 4, 0), ("couette", 7, 1), ("sphere", 5, 2),
                                             ("pipe", 12, 0)])
@pytest.mark.parametrize("scheme", [(0, 1, 0, 1.0), (0, 1, 1, 0.7)])
def test_fp64_adjoint_equals_oracle_adjoint(kind, steps, ckpt, scheme):
    w = _case(kind)
    rho, u, mask, ut = _inputs(w, 7)
    lat = OL.BY_NAME[w["lattice"]]
    o = O.Simulation(lat, w["shape"], w["S"], 1.0, w["solid"], w["links"], scheme=scheme,
                     force=w["force"], skew=w.get("skew", (0, 0)))
    o.init_equilibrium(rho, u)
    J0, gs0, gq0, gp0 = OA.adjoint(o, steps, mask, ut)
    g = gpu_sim(w, "f64", scheme=scheme)
    g.init_equilibrium(rho, u)
    J, gs, gq, gp = g.adjoint(steps, mask, ut, checkpoint_every=ckpt)
    assert abs(J - J0) <= 1e-12 * abs(J0)
    scale = max(np.abs(gs0).max(), np.abs(gq0).max(), np.abs(gp0).max())
    assert np.abs(gs - gs0).max() <= 1e-10 * scale
    assert np.abs(gq - gq0).max() <= 1e-10 * scale
    assert np.abs(gp[:, : lat.D] - gp0[:, : lat.D]).max() <= 1e-10 * scale
    # the context ends in the state after the forward run
    assert g.time() == steps
    ref = gpu_sim(w, "f64", scheme=scheme)
    ref.init_equilibrium(rho, u)
    ref.step(steps)
    fl = ~w["solid"]
    assert np.array_equal(g.get_populations()[:, fl], ref.get_populations()[:, fl])


def test_fp64_adjoint_vs_central_differences_sphere():
    """32^3 periodic box with a sphere, 40 steps, body force: dJ/ds_nu (sum over the
    viscous rows), dJ/dq and dJ/dphi of sampled links against central differences
    of the GPU forward run with h = 1e-4."""
    w = W.sphere_3d(32, 5.2, (16.37, 15.71, 16.13), s_nu=1.0, force=(1e-5, 0.0, 0.0))
    N = 32 ** 3
    x = np.arange(N) % 32
    mask = (x >= 22) & (x < 26)
    rng = np.random.default_rng(5)
    ut = 1e-4 * rng.standard_normal((N, 3))
    steps = 40
    base = gpu_sim(w, "f64")
    base.init_equilibrium()
    f0 = base.get_populations()
    J, gs, gq, gp = base.adjoint(steps, mask, ut)
    viscous = [9, 11, 13, 14, 15]

    def J_of(s=None, q=None, uw=None):
        sim = gpu_sim(w, "f64")
        if s is not None:
            sim.set_relaxation(s)
        if q is not None or uw is not None:
            sim.set_link_values(q, uw)
        sim.set_populations(f0)
        return sim.adjoint(steps, mask, ut)[0]

    h = 1e-4
    scale = max(np.abs(gs).max(), np.abs(gq).max(), np.abs(gp).max())
    S = w["S"].copy()
    sp, sm = S.copy(), S.copy()
    sp[viscous] += h
    sm[viscous] -= h
    fd = (J_of(s=sp) - J_of(s=sm)) / (2 * h)
    assert abs(fd - gs[viscous].sum()) <= 1e-4 * max(abs(fd), scale)
    q0 = w["links"]["q"].copy()
    uw0 = np.zeros((len(q0), 3))
    for k in rng.choice(len(q0), 4, replace=False):
        qp, qm = q0.copy(), q0.copy()
        qp[k] = min(q0[k] + h, 1.0)
        qm[k] = q0[k] - h
        fd = (J_of(q=qp) - J_of(q=qm)) / (qp[k] - qm[k])
        assert abs(fd - gq[k]) <= 1e-4 * scale
        for a in range(3):
            up, um = uw0.copy(), uw0.copy()
            up[k, a] += h
            um[k, a] -= h
            fd = (J_of(uw=up) - J_of(uw=um)) / (2 * h)
            assert abs(fd - gp[k, a]) <= 1e-4 * scale


def test_fp32_adjoint_close_to_fp64():
    w = _case("pipe")
    rho, u, mask, ut = _inputs(w, 11)
    res = {}
    for prec in ("f64", "f32"):
        g = gpu_sim(w, prec)
        g.init_equilibrium(rho, u)
        res[prec] = g.adjoint(20, mask, ut)
    J64, gs64, gq64, gp64 = res["f64"]
    J32, gs32, gq32, gp32 = res["f32"]
    scale = max(np.abs(gs64).max(), np.abs(gq64).max(), np.abs(gp64).max())
    assert abs(J32 - J64) <= 1e-3 * J64
    for a, b in ((gs32, gs64), (gq32, gq64), (gp32, gp64)):
        err = np.abs(a - b).max() / scale
        print("fp32 adjoint gradient error %.3e" % err)
        assert err <= 1e-3


def test_autograd_function():
    torch = pytest.importorskip("torch")
    w = _case("couette")
    rho, u, mask, ut = _inputs(w, 13)
    sim = gpu_sim(w, "f64")
    sim.init_equilibrium(rho, u)
    f0 = sim.get_populations()
    F = B.adjoint_loss_function()
    q = torch.tensor(w["links"]["q"], requires_grad=True)
    s = torch.tensor(w["S"], requires_grad=True)
    uw = torch.tensor(w["links"]["uw"], requires_grad=True)
    J = F.apply(q, s, uw, sim, f0, 6, mask, ut, 0)
    (3.0 * J).backward()
    ref = gpu_sim(w, "f64")
    ref.init_equilibrium(rho, u)
    J0, gs, gq, gp = ref.adjoint(6, mask, ut)
    assert abs(J.item() - J0) <= 1e-14 * J0
    assert np.allclose(q.grad.numpy(), 3 * gq, rtol=0, atol=1e-15 + 1e-13 * np.abs(gq).max())
    assert np.allclose(s.grad.numpy(), 3 * gs, rtol=0, atol=1e-15 + 1e-13 * np.abs(gs).max())
    assert np.allclose(uw.grad.numpy(), 3 * gp, rtol=0, atol=1e-15 + 1e-13 * np.abs(gp).max())


@pytest.mark.parametrize("prec,tol", [("f64", 1e-6), ("f32", 2e-3)])
def test_adjoint_ds_vs_central_differences_large_grid(prec, tol):
    """An 80^3 periodic box (512,000 nodes, many thread blocks per SM) with a sphere:
    dJ/ds_nu summed over the viscous rows against central differences of the FP64
    forward run with h = 1e-4.  Catches per-block or per-thread accumulation that
    drops nodes on large grids."""
    w = W.sphere_3d(80, 12.5, (40.3, 39.8, 40.6), s_nu=1.0, force=(1e-5, 0.0, 0.0))
    N = 80 ** 3
    x = np.arange(N) % 80
    mask = (x >= 60) & (x < 66)
    rng = np.random.default_rng(21)
    ut = 1e-4 * rng.standard_normal((N, 3))
    steps = 30
    viscous = [9, 11, 13, 14, 15]
    sim = gpu_sim(w, prec)
    sim.init_equilibrium()
    J, gs, gq, gp = sim.adjoint(steps, mask, ut)

    def J_of(sv):
        s2 = gpu_sim(w, "f64")
        S = w["S"].copy()
        S[viscous] = sv
        s2.set_relaxation(S)
        s2.init_equilibrium()
        return s2.adjoint(steps, mask, ut)[0]

    h = 1e-4
    fd = (J_of(1.0 + h) - J_of(1.0 - h)) / (2 * h)
    assert abs(gs[viscous].sum() - fd) <= tol * abs(fd)


def test_bf16_storage_adjoint_recomputes_with_the_sweep():
    """16-bit storage recomputes segments with the sweep itself (raw checkpoints):
    the gradients stay close to the FP64 adjoint's (BF16 rounds every step)."""
    w = _case("pipe")
    rho, u, mask, ut = _inputs(w, 11)
    res = {}
    for prec in ("f64", "bf16"):
        g = gpu_sim(w, prec)
        g.init_equilibrium(rho, u)
        res[prec] = g.adjoint(20, mask, ut, checkpoint_every=6)
    J64, gs64, gq64, gp64 = res["f64"]
    J16, gs16, gq16, gp16 = res["bf16"]
    scale = max(np.abs(gs64).max(), np.abs(gq64).max(), np.abs(gp64).max())
    errs = [np.abs(a - b).max() / scale for a, b in ((gs16, gs64), (gq16, gq64), (gp16, gp64))]
    print("bf16 adjoint: J %.3e vs %.3e, gradient errors %s" % (J16, J64, errs))
    assert abs(J16 - J64) <= 0.2 * J64
    assert max(errs) <= 0.2
