"""The two-node variant of the scheme (Sec. 2, Remark (2), Eq. 2.11) through the
C-ABI (lbm_set_two_node) against the oracle's two-node option: element-wise FP64
parity in 2D and 3D, a reduced-precision bound, second order on the Poiseuille
channel, and the calls that must refuse it."""

import numpy as np
import pytest

from oracle import lattices as OL
from oracle import lbm as O
from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import check_close, deviation, gpu_sim, require_gpu

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _pair(w, scheme, prec="f64"):
    lat = OL.BY_NAME[w["lattice"]]
    o = O.Simulation(lat, w["shape"], w["S"], w.get("rho0", 1.0), w["solid"], w["links"],
                     scheme=scheme, force=w.get("force", (0.0, 0.0, 0.0)),
                     skew=w.get("skew", (0, 0)), two_node=True)
    g = gpu_sim(w, prec, scheme=scheme)
    g.set_two_node(True)
    return lat, o, g


@pytest.mark.parametrize("scheme", [(0, 1, 0, 1.0), (0, 1, 1, 0.7), (0, 0, 1, 1.0)])
@pytest.mark.parametrize("steps", [1, 2, 37])
def test_couette_two_node_matches_oracle(scheme, steps):
    w = W.couette_config(64)
    w["links"] = W.random_links_uw(w["links"], 0.01, seed=2)
    rho, u = W.random_state(w["shape"], "D2Q9", 1.0, 0.01, seed=3)
    lat, o, g = _pair(w, scheme)
    o.init_equilibrium(rho, u)
    g.init_equilibrium(rho, u)
    o.step(steps)
    g.step(steps)
    fl = ~w["solid"]
    check_close(deviation(g.get_populations(), lat), deviation(o.f, lat), TOL64, fl)


@pytest.mark.parametrize("lattice", ["D3Q19", "D3Q15"])
def test_sphere_and_pipe_two_node_match_oracle(lattice):
    """A sphere box (x_l solid for some links: they keep Eq. 2.10) and the skewed pipe."""
    for w in (W.sphere_3d(12, 3.1, (5.7, 6.2, 5.4), s_nu=1.1, force=(1e-5, 0.0, 2e-6), lattice=lattice),
              W.tilted_pipe_3d(16, lattice=lattice)):
        w["links"] = W.random_links_uw(w["links"], 0.01, seed=4)
        rho, u = W.random_state(w["shape"], lattice, 1.0, 0.005, seed=5)
        lat, o, g = _pair(w, (0, 1, 1, 0.8))
        o.init_equilibrium(rho, u)
        g.init_equilibrium(rho, u)
        o.step(13)
        g.step(13)
        fl = ~w["solid"]
        check_close(deviation(g.get_populations(), lat), deviation(o.f, lat), TOL64, fl)


def test_fp32_two_node_bound():
    w = W.couette_config(64)
    lat, o, g = _pair(w, (0, 1, 0, 1.0), prec="f32")
    o.init_equilibrium()
    g.init_equilibrium()
    o.step(3000)
    g.step(3000)
    fl = ~w["solid"]
    _, ug = g.moments()
    _, uo = o.moments()
    check_close(ug[fl][:, :2], uo[fl][:, :2], 2e-6, None, "two-node f32 u")


def test_two_node_poiseuille_second_order_and_switching_off():
    sizes = [11, 21, 41]
    errs = []
    for n in sizes:
        w = W.poiseuille_2d(n, 0.75, 1.0)
        g = gpu_sim(w, "f64", scheme=(0, 1, 1, 1.0))
        g.set_two_node(True)
        ue = np.nan_to_num(w["u_exact"])
        g.init_equilibrium(None, ue)
        g.step(int(12 * n * n / (np.pi ** 2 / 6)) // 2 * 2)
        errs.append(g.error_norms(ue)["l2_rel"])
    inv_h = [n - 2 + 1.5 for n in sizes]
    p = -np.polyfit(np.log(inv_h), np.log(errs), 1)[0]
    print("two-node Poiseuille E_r", errs, "order", p)
    assert 1.85 < p < 2.4
    # switched off again, a context steps exactly like one that never had it
    w = W.couette_config(64)
    a, b = gpu_sim(w, "f64"), gpu_sim(w, "f64")
    a.set_two_node(True)
    a.set_two_node(False)
    a.init_equilibrium()
    b.init_equilibrium()
    a.step(25)
    b.step(25)
    fl = ~w["solid"]
    assert np.array_equal(a.get_populations()[:, fl], b.get_populations()[:, fl])


def test_adjoint_and_batch_refuse_two_node():
    w = W.couette_config(32)
    g = gpu_sim(w, "f64")
    g.set_two_node(True)
    g.init_equilibrium()
    N = 32 * 32
    with pytest.raises(B.LbmError) as ei:
        g.adjoint(3, np.ones(N, bool), np.zeros((N, 2)))
    assert ei.value.code == -7
    batch = B.Batch([g])
    with pytest.raises(B.LbmError) as ei:
        batch.step(2)
    assert ei.value.code == -7
    batch.close()
