"""Pins of the oracle's discrete adjoint against central finite differences of the
oracle's own forward run (the adjoint is exact for the discrete map, so the two
agree to the finite-difference truncation)."""

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import lattices as L
from oracle import lbm as O
from paper_1712_08288_gb300 import workloads as W


def _case_2d():
    w = W.couette_2d(14, (7.2, 6.9), 2.1, 6.1, 0.01)
    w["links"] = W.random_links_uw(w["links"], 0.01, seed=1)
    rng = np.random.default_rng(2)
    w["links"]["q"] = rng.uniform(0.1, 1.0, len(w["links"]["q"]))
    S = W.relaxation_rates("D2Q9", 1.3)
    return L.D2Q9, w, S, (2e-5, -1e-5, 0.0)


def _case_3d():
    w = W.sphere_3d(6, 1.7, (2.6, 3.1, 2.4), s_nu=1.1)
    w["links"] = W.random_links_uw(w["links"], 0.01, seed=3)
    S = W.relaxation_rates("D3Q19", 1.1)
    return L.D3Q19, w, S, (1e-5, 0.0, 2e-5)


def _case_3d_q15():
    w = W.sphere_3d(6, 1.7, (2.6, 3.1, 2.4), s_nu=1.1, lattice="D3Q15")
    w["links"] = W.random_links_uw(w["links"], 0.01, seed=5)
    S = W.relaxation_rates("D3Q15", 1.1)
    return L.D3Q15, w, S, (1e-5, 2e-5, 0.0)


def _run(lat, w, S, g, scheme, links, steps, mask, ut, rho, u, grad):
    sim = O.Simulation(lat, w["shape"], S, 1.0, w["solid"], links, scheme=scheme, force=g)
    sim.init_equilibrium(rho, u)
    return A.adjoint(sim, steps, mask, ut) if grad else A.loss(sim, steps, mask, ut)


@pytest.mark.parametrize("case", [_case_2d, _case_3d, _case_3d_q15])
@pytest.mark.parametrize("scheme", [(0, 1, 0, 1.0), (0, 1, 1, 0.7)])
def test_adjoint_matches_finite_differences(case, scheme):
    lat, w, S, g = case()
    N = w["shape"][0] * w["shape"][1] * w["shape"][2]
    D = lat.D
    rng = np.random.default_rng(7)
    rho, u = W.random_state(w["shape"], lat.name, 1.0, 0.01, seed=8)
    mask = rng.random(N) < 0.5
    ut = 0.01 * rng.standard_normal((N, D))
    steps = 4
    links = w["links"]
    J, gs, gq, gphi = _run(lat, w, S, g, scheme, links, steps, mask, ut, rho, u, True)
    h = 1e-6

    def fd(modify):
        lp, sp = modify(+h)
        jp = _run(lat, w, sp, g, scheme, lp, steps, mask, ut, rho, u, False)
        lm, sm = modify(-h)
        jm = _run(lat, w, sm, g, scheme, lm, steps, mask, ut, rho, u, False)
        return (jp - jm) / (2 * h)

    scale = np.abs(np.concatenate([gs, gq, gphi.ravel()])).max()
    for k in [1, 2, lat.Q - 1, lat.Q - 2]:                # non-conserved rates
        def mod(e, k=k):
            s2 = S.copy()
            s2[k] += e
            return links, s2
        assert abs(fd(mod) - gs[k]) < 1e-6 * scale, ("s", k)
    for k in [0, len(gq) // 2, len(gq) - 1]:
        def modq(e, k=k):
            l2 = dict(links)
            l2["q"] = links["q"].copy()
            l2["q"][k] += e
            return l2, S
        assert abs(fd(modq) - gq[k]) < 1e-6 * scale, ("q", k)
        for a in range(D):
            def modp(e, k=k, a=a):
                l2 = dict(links)
                l2["uw"] = links["uw"].copy()
                l2["uw"][k, a] += e
                return l2, S
            assert abs(fd(modp) - gphi[k, a]) < 1e-6 * scale, ("phi", k, a)
    # conserved rows have no influence
    for k in [0] + list(lat.j_rows):
        assert abs(gs[k]) < 1e-12 * scale
