"""Convergence under grid refinement on the GPU: the circular Couette problem (curved
walls, the 64^2 configuration scaled with n in diffusive scaling) run to steady
state through the C-ABI.  The paper states second order for the single-node scheme
on curved walls (Sec. 3); the bar here is an observed order of at least 1.9 in FP64,
with FP32 deviation storage reaching the same error (within 5 %) after the same
number of steps."""

import numpy as np
import pytest

from paper_1712_08288_gb300 import workloads as W

from gpu_common import check_fd, gpu_sim, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _steady(w, prec, tol, steps=None, chunk=200, max_steps=400000):
    ue = np.nan_to_num(w["u_exact"])
    sim = gpu_sim(w, prec)
    sim.init_equilibrium(None, ue)
    if steps is None:
        sim.error_norms(ue)
        steps, res = 0, 1.0
        while res >= tol:
            assert steps < max_steps, "no steady state"
            sim.step(chunk)
            steps += chunk
            res = sim.error_norms(ue)["residual"]
    else:
        sim.step(steps)
    return sim.error_norms(ue)["l2_rel"], steps


def test_couette_refinement_order_fp64_and_fp32():
    sizes = [32, 64, 128]
    e64, e32 = [], []
    for n in sizes:
        w = W.couette_config(n)
        e, steps = _steady(w, "f64", 1e-10)
        e64.append(e)
        e32.append(_steady(w, "f32", None, steps=steps)[0])
    order = -np.polyfit(np.log(sizes), np.log(e64), 1)[0]
    print("E_r f64", e64, "f32", e32, "order", order)
    assert order >= 1.9, (e64, order)
    for a, b in zip(e32, e64):
        assert abs(a - b) <= 0.05 * b


RULES = {"g": (0, 1, 0), "1.5g": (0, 1.5, 0), "2g": (0, 2, 0), "g2": (0, 0, 1), "g2+g": (0, 1, 1)}


@pytest.mark.parametrize("s_nu", [0.5, 1.0, 1.5, 1.99])
def test_poiseuille_parameter_grid_second_order(s_nu):
    """The paper's Poiseuille grid (Sec. 3.1): the five l-rules x gamma in {0.25, 0.75,
    1} at one s_nu, N_y = 11, 21, 41, all 45 channels advanced together as one
    batch (one launch per step) from the analytic start for 12 diffusion times of the
    widest channel.  Every (rule, gamma) shows an observed order between 1.8 and 2.5
    (Sec. 3.1 reports orders near 2 for all of them)."""
    from paper_1712_08288_gb300 import binding as B
    sizes = [11, 21, 41]
    cases = [(r, gm, n) for r in RULES for gm in (0.25, 0.75, 1.0) for n in sizes]
    sims, ws = [], []
    for r, gm, n in cases:
        w = W.poiseuille_2d(n, gm, s_nu)
        sim = gpu_sim(w, "f64", scheme=RULES[r] + (1.0,))
        sim.init_equilibrium(None, np.nan_to_num(w["u_exact"]))
        sims.append(sim)
        ws.append(w)
    nu = (1.0 / s_nu - 0.5) / 3.0
    tau = (max(sizes) ** 2) / (np.pi ** 2 * nu)
    steps = 2 * int(6 * tau)
    batch = B.Batch(sims)
    batch.step(steps)
    batch.close()
    errs = {}
    for (r, gm, n), sim, w in zip(cases, sims, ws):
        errs.setdefault((r, gm), []).append(sim.error_norms(np.nan_to_num(w["u_exact"]))["l2_rel"])
    bad = {}
    for (r, gm), e in errs.items():
        inv_h = [n - 2 + 2 * gm for n in sizes]
        p = -np.polyfit(np.log(inv_h), np.log(e), 1)[0]
        print("s_nu %.2f rule %-5s gamma %.2f E_r %s order %.2f" % (s_nu, r, gm, e, p))
        if not 1.8 < p < 2.5:
            bad[(r, gm)] = (e, p)
    assert not bad, bad


def _tg_gpu(w, rule, prec="f64"):
    sim = gpu_sim(w, prec, scheme=RULES[rule] + (1.0,))
    sim.init_equilibrium(w["rho_init"], np.nan_to_num(w["u_exact"]))
    sim.set_wall_factor(1.0, w["decay"])
    return sim


def test_taylor_green_moving_wall_matches_oracle():
    """The moving curved wall of Sec. 3.2 (wall velocity decaying every step through
    lbm_set_wall_factor) against the oracle with phi(x_b, t) reset before each step."""
    from oracle import lattices as OL
    from oracle import lbm as O
    from gpu_common import check_close, deviation
    w = W.taylor_green_disc(40, 1.0)
    o = O.Simulation(OL.D2Q9, w["shape"], w["S"], 1.0, w["solid"], w["links"],
                     scheme=RULES["g2+g"] + (1.0,))
    o.init_equilibrium(w["rho_init"], np.nan_to_num(w["u_exact"])[:, :2])
    uw0 = w["links"]["uw"].copy()
    steps = 61
    for n in range(steps):
        o.link_uw = uw0 * w["decay"] ** n
        o.step()
    g = _tg_gpu(w, "g2+g")
    g.step(steps)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), OL.D2Q9), deviation(o.f, OL.D2Q9), 1e-12, fl)


@pytest.mark.parametrize("s_nu", [0.5, 1.0, 1.5, 1.99])
def test_taylor_green_disc_second_order(s_nu):
    """Sec. 3.2: E_r at T = 1/U0 for h = 1/40 and 1/80, all five l-rules; second
    order (ratio of errors about 4) at every s_nu including 1.99."""
    bad = {}
    for rule in RULES:
        e = []
        for inv_h in (40, 80):
            w = W.taylor_green_disc(inv_h, s_nu)
            sim = _tg_gpu(w, rule)
            sim.step(w["steps"])
            ue = np.nan_to_num(w["u_exact"]) * w["decay"] ** w["steps"]
            e.append(sim.error_norms(ue)["l2_rel"])
        p = np.log(e[0] / e[1]) / np.log(2)
        print("TG s_nu %.2f rule %-5s E_r %s order %.2f" % (s_nu, rule, e, p))
        if not 1.7 < p < 2.8:
            bad[rule] = (e, p)
    assert not bad, bad


def test_adjoint_follows_the_wall_factor():
    """dJ/dq and dJ/dphi with a decaying wall velocity against central differences
    of the forward run (FP64)."""
    w = W.taylor_green_disc(40, 1.0)
    N = w["shape"][0] * w["shape"][1]
    rng = np.random.default_rng(31)
    mask = rng.random(N) < 0.5
    ut = np.zeros((N, 2))
    steps = 40

    def run(q=None, uw=None, grad=False):
        sim = gpu_sim(w, "f64", scheme=RULES["g"] + (1.0,))
        if q is not None or uw is not None:
            sim.set_link_values(q, uw)
        sim.init_equilibrium(w["rho_init"], np.nan_to_num(w["u_exact"]))
        sim.set_wall_factor(1.0, w["decay"] ** 20)      # a strong decay to test the weighting
        return sim.adjoint(steps, mask, ut)

    J, gs, gq, gp = run()
    q0 = w["links"]["q"].copy()
    uw0 = w["links"]["uw"].copy()
    h = 1e-6
    floor = 1e-12 * abs(J) / h      # rounding of two FP64 evaluations of J over 2h
    for k in rng.choice(len(q0), 3, replace=False):
        qp, qm = q0.copy(), q0.copy()
        qp[k] = min(q0[k] + h, 1.0)
        qm[k] = q0[k] - h
        fd = (run(q=qp)[0] - run(q=qm)[0]) / (qp[k] - qm[k])
        check_fd(fd, gq[k], 1e-5, floor, "TG dJ/dq[%d]" % k)
        for a in range(2):
            up, um = uw0.copy(), uw0.copy()
            up[k, a] += h
            um[k, a] -= h
            fd = (run(uw=up)[0] - run(uw=um)[0]) / (2 * h)
            check_fd(fd, gp[k, a], 1e-5, floor, "TG dJ/dphi[%d,%d]" % (k, a))
