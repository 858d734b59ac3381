"""Convergence under grid refinement on the GPU: the circular Couette problem (curved
walls, the 64^2 configuration scaled with n in diffusive scaling) run to steady
state through the C-ABI.  The paper states second order for the single-node scheme
on curved walls (Sec. 3); the bar here is an observed order of at least 1.9 in FP64,
with FP32 deviation storage reaching the same error (within 5 %) after the same
number of steps."""

import numpy as np
import pytest

from paper_1712_08288_gb300 import workloads as W

from gpu_common import gpu_sim, require_gpu

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
