"""Failure detection through the C-ABI, with every fault made on the host: a NaN
written into the populations with lbm_set_populations (the sweep's status word then
reports LBM_EDIVERGED at the next read-out, and a new initial state clears it),
invalid inputs rejected before any launch.  Nothing here
faults, traps or hangs the GPU."""

import numpy as np
import pytest

from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import gpu_sim, require_gpu

pytestmark = pytest.mark.gpu

EINVAL, ENONCONVEX, EDIVERGED, ETIMEOUT = -1, -4, -5, -6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _code(fn):
    with pytest.raises(B.LbmError) as ei:
        fn()
    return ei.value.code


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_nan_population_is_reported_as_diverged(prec):
    w = W.couette_config(32)
    g = gpu_sim(w, prec)
    g.init_equilibrium()
    f = g.get_populations()
    fl = np.nonzero(~w["solid"])[0]
    f[3, fl[len(fl) // 2]] = np.nan
    g.set_populations(f)
    g.step(2)
    assert _code(lambda: g.error_norms()) == EDIVERGED
    assert _code(lambda: g.moments()) == EDIVERGED
    # a fresh initial state clears the status word; the run is healthy again
    g.init_equilibrium()
    g.step(4)
    assert g.error_norms()["status"] == 0
    _, u = g.moments()
    assert np.all(np.isfinite(u[fl]))


def test_invalid_inputs_are_rejected_before_any_launch():
    w = W.couette_config(32)
    S = w["S"]
    # bad lattice, grid, rates
    assert _code(lambda: B.Lbm("D2Q9", (32, 32, 2), S)) == EINVAL
    assert _code(lambda: B.Lbm("D2Q9", (0, 32, 1), S)) == EINVAL
    bad = S.copy()
    bad[7] = 2.5
    assert _code(lambda: B.Lbm("D2Q9", (32, 32, 1), bad)) == EINVAL
    g = B.Lbm("D2Q9", (32, 32, 1), S)
    # a new context is an all-fluid periodic box: it steps, and keeps its mass
    g.init_equilibrium()
    m0 = g.error_norms()["mass"]
    g.step(3)
    assert abs(g.error_norms()["mass"] - m0) < 1e-12 * abs(m0)
    # skew out of range
    assert _code(lambda: g.set_skew(32, 0)) == EINVAL
    # wall fraction outside (0, 1]
    links = dict(w["links"])
    links["q"] = links["q"].copy()
    links["q"][0] = 1.5
    assert _code(lambda: g.set_geometry(w["solid"], links)) == EINVAL
    links["q"][0] = 0.0
    assert _code(lambda: g.set_geometry(w["solid"], links)) == EINVAL
    # a link list that does not match the solid flags
    links = {k: v[1:] for k, v in w["links"].items()}
    assert _code(lambda: g.set_geometry(w["solid"], links)) == EINVAL
    g.set_geometry(w["solid"], w["links"])
    # Eq. 2.12: l = 0 is non-convex for gamma > 1/2 unless allowed
    assert _code(lambda: g.set_scheme(0, 0, 0, 1.0)) == ENONCONVEX
    g.set_scheme(0, 0, 0, 1.0, allow_nonconvex=True)
    assert _code(lambda: g.set_scheme(0, 1, 0, 0.0)) == EINVAL       # b outside (0, 1]
    assert _code(lambda: g.set_scheme(-1, 0, 0, 1.0)) == EINVAL      # l < 0
    assert _code(lambda: g.set_wall_factor(1.0, 0.0)) == EINVAL
    assert _code(lambda: g.step(-1)) == EINVAL
    g.step(0)                                                        # nothing to do
    assert g.time() == 0


@pytest.mark.parametrize("lattice,prec", [("D2Q9", "f32"), ("D3Q19", "f64"), ("D3Q19", "bf16")])
def test_bounded_wait_gives_up_and_reports_timeout(lattice, prec):
    """The sweep's bounded wait, made to run out on the host's say: with a wait
    limit of zero polls every warp gives up at its first tile (after waiting, with
    the default limit, for its own copies in flight), the step leaves the
    populations untouched and the next read-out reports LBM_ETIMEOUT.  With the
    default limit back and a new initial state the context steps like a fresh one."""
    w = W.couette_config(48) if lattice == "D2Q9" else W.tilted_pipe_3d(32)
    u0 = np.nan_to_num(w["u_exact"])
    g = gpu_sim(w, prec)
    g.init_equilibrium(None, u0)
    f0 = g.get_populations()
    g.set_wait_limit(0)
    g.step(2)                      # an even count: the layout parity is unchanged
    assert _code(lambda: g.moments()) == ETIMEOUT
    assert _code(lambda: g.error_norms()) == ETIMEOUT
    fl = ~w["solid"]
    assert np.array_equal(g.get_populations()[:, fl], f0[:, fl])   # no tile was processed
    assert _code(lambda: g.set_wait_limit(-1)) == EINVAL
    g.set_wait_limit(1000)
    g.init_equilibrium(None, u0)
    g.step(6)
    ref = gpu_sim(w, prec)
    ref.init_equilibrium(None, u0)
    ref.step(6)
    assert g.error_norms()["status"] == 0
    assert np.array_equal(g.get_populations()[:, fl], ref.get_populations()[:, fl])
