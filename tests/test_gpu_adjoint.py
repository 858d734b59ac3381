"""GPU discrete adjoint (lbm_adjoint) against the oracle's FP64 discrete adjoint and
against central finite differences of the GPU forward run.

Tolerances: FP64 GPU vs oracle adjoint 1e-10 relative to the largest gradient
(different summation order over nodes and steps); FP64 adjoint vs central
differences with h = 1e-4: every checked entry within 1e-4 of its own difference
quotient, above the quotient's rounding floor (1e-12 |J| / h); FP32 adjoint vs
FP64 adjoint 1e-3 (measured and stated in the design notes)."""

import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import lattices as OL
from oracle import lbm as O
from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import check_close, check_fd, gpu_sim, require_gpu

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
    # every gradient entry within 1e-10 of the largest gradient of its own kind
    check_close(gs, gs0, 1e-10, None, "dJ/ds")
    check_close(gq, gq0, 1e-10, None, "dJ/dq")
    check_close(gp[:, : lat.D], gp0[:, : lat.D], 1e-10, None, "dJ/dphi")
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
    # each entry within 1e-4 of its own central difference, above the quotient's
    # rounding floor: two FP64 evaluations of J, each good to ~1e-12 |J|, over 2h
    floor = 1e-12 * abs(J) / h
    S = w["S"].copy()
    sp, sm = S.copy(), S.copy()
    sp[viscous] += h
    sm[viscous] -= h
    fd = (J_of(s=sp) - J_of(s=sm)) / (2 * h)
    check_fd(fd, gs[viscous].sum(), 1e-4, floor, "dJ/ds_nu")
    q0 = w["links"]["q"].copy()
    uw0 = np.zeros((len(q0), 3))
    for k in rng.choice(len(q0), 4, replace=False):
        qp, qm = q0.copy(), q0.copy()
        qp[k] = min(q0[k] + h, 1.0)
        qm[k] = q0[k] - h
        fd = (J_of(q=qp) - J_of(q=qm)) / (qp[k] - qm[k])
        check_fd(fd, gq[k], 1e-4, floor, "dJ/dq[%d]" % k)
        for a in range(3):
            up, um = uw0.copy(), uw0.copy()
            up[k, a] += h
            um[k, a] -= h
            fd = (J_of(uw=up) - J_of(uw=um)) / (2 * h)
            check_fd(fd, gp[k, a], 1e-4, floor, "dJ/dphi[%d,%d]" % (k, a))


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


@pytest.mark.parametrize("device", ["cpu", "cuda"])
def test_autograd_function(device):
    """The autograd Function's forward runs only the checkpointed forward pass
    (lbm_adjoint_forward), its backward the recompute and adjoint sweep
    (lbm_adjoint_backward); the gradients equal lbm_adjoint's, arrive on the
    inputs' device and dtype, and a backward after the context was stepped in
    between is refused."""
    torch = pytest.importorskip("torch")
    w = _case("couette")
    rho, u, mask, ut = _inputs(w, 13)
    sim = gpu_sim(w, "f64")
    sim.init_equilibrium(rho, u)
    f0 = sim.get_populations()
    F = B.adjoint_loss_function()
    q = torch.tensor(w["links"]["q"], device=device, requires_grad=True)
    s = torch.tensor(w["S"], device=device, requires_grad=True)
    uw = torch.tensor(w["links"]["uw"], device=device, requires_grad=True)
    J = F.apply(q, s, uw, sim, f0, 6, mask, ut, 0)
    assert J.device == q.device
    assert sim.time() == 6                      # the forward pass ran the 6 steps only
    (3.0 * J).backward()
    ref = gpu_sim(w, "f64")
    ref.init_equilibrium(rho, u)
    J0, gs, gq, gp = ref.adjoint(6, mask, ut)
    assert abs(J.item() - J0) <= 1e-14 * J0
    for t, want in ((q, gq), (s, gs), (uw, gp)):
        assert t.grad.device == t.device and t.grad.dtype == t.dtype
        assert np.allclose(t.grad.cpu().numpy(), 3 * want, rtol=0, atol=1e-15 + 1e-13 * np.abs(want).max())
    # the tape is gone once the context steps between forward and backward
    J = F.apply(q, s, uw, sim, f0, 6, mask, ut, 0)
    sim.step(1)
    with pytest.raises(B.LbmError) as ei:
        J.backward()
    assert ei.value.code == -7


def test_split_adjoint_equals_lbm_adjoint_and_backward_repeats():
    """lbm_adjoint_forward + lbm_adjoint_backward give lbm_adjoint's gradients bit
    for bit and its loss to rounding (FP64, FP32 and BF16 storage, with
    checkpointing), the context ends in the forward end state, and a second
    backward pass repeats the first to the recomputation's rounding."""
    w = _case("pipe")
    rho, u, mask, ut = _inputs(w, 17)
    for prec in ("f64", "f32", "bf16"):
        a = gpu_sim(w, prec)
        a.init_equilibrium(rho, u)
        J0, gs0, gq0, gp0 = a.adjoint(14, mask, ut, checkpoint_every=4)
        b = gpu_sim(w, prec)
        b.init_equilibrium(rho, u)
        J = b.adjoint_forward(14, mask, ut, checkpoint_every=4)
        assert b.time() == 14 and abs(J - J0) <= 1e-14 * abs(J0)   # J: atomic sum order
        gs, gq, gp = b.adjoint_backward()
        assert np.array_equal(gs, gs0) and np.array_equal(gq, gq0) and np.array_equal(gp, gp0)
        assert b.time() == 14
        # a repeated backward pass recomputes the last segment too (the first used
        # the states the forward sweep saved): FP64 and FP32 storage recompute with
        # the push-form step, whose rounding differs from the sweep's in FP32
        gs2, gq2, gp2 = b.adjoint_backward()
        tol = {"f64": 1e-12, "f32": 1e-5, "bf16": 0.0}[prec]
        for x2, x0 in ((gs2, gs0), (gq2, gq0), (gp2, gp0)):
            assert np.abs(x2 - x0).max() <= tol * np.abs(x0).max()
        assert b.time() == 14
        fl = ~w["solid"]
        assert np.array_equal(a.get_populations()[:, fl], b.get_populations()[:, fl])
    with pytest.raises(B.LbmError) as ei:
        gpu_sim(w, "f64").adjoint_backward()       # no forward pass on this context
    assert ei.value.code == -7


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


def test_fd_links_full_size_sphere_128():
    """The adjoint case at its full size: a sphere of radius 20 in a periodic 128^3
    box, body force 1e-6 along x, 2000 steps from rest, FP64, J over the slab
    96 <= x < 104.  dJ/dq of 16 links (the 8 with the largest gradient and 8 drawn
    at random) and, for the same links, the derivative of J along a random unit
    change of the wall velocity, against central differences (h = 1e-4): each within
    1e-4 of its own difference quotient, above the quotient's rounding floor."""
    n, K = 128, 2000
    w = W.sphere_3d(n, 20.0, (64.37, 63.71, 64.13), s_nu=1.0, force=(1e-6, 0.0, 0.0))
    N = n ** 3
    x = np.arange(N) % n
    mask = (x >= 96) & (x < 104)
    rng = np.random.default_rng(41)
    ut = 1e-6 * rng.standard_normal((N, 3))
    sim = gpu_sim(w, "f64")
    sim.init_equilibrium()
    J, gs, gq, gp = sim.adjoint(K, mask, ut)
    q0 = w["links"]["q"].copy()
    uw0 = np.zeros((len(q0), 3))
    top = np.argsort(-np.abs(gq))[:8]
    rest = np.setdiff1d(np.arange(len(q0)), top)
    links = np.concatenate([top, rng.choice(rest, 8, replace=False)])

    def J_of(q=None, uw=None):
        sim.set_link_values(q if q is not None else q0, uw if uw is not None else uw0)
        sim.init_equilibrium()
        return sim.adjoint_forward(K, mask, ut)

    h = 1e-4
    floor = 1e-12 * abs(J) / h
    for k in links:
        qp, qm = q0.copy(), q0.copy()
        qp[k] = min(q0[k] + h, 1.0)
        qm[k] = q0[k] - h
        fd = (J_of(q=qp) - J_of(q=qm)) / (qp[k] - qm[k])
        check_fd(fd, gq[k], 1e-4, floor, "128^3 dJ/dq[%d]" % k)
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        up, um = uw0.copy(), uw0.copy()
        up[k] += h * v
        um[k] -= h * v
        fd = (J_of(uw=up) - J_of(uw=um)) / (2 * h)
        check_fd(fd, float(gp[k] @ v), 1e-4, floor, "128^3 dJ/dphi[%d].v" % k)
