"""Pins of the oracle's boundary scheme (Sec. 2 of arXiv:1712.08288) against the
closed forms and special cases the paper states, and against a separately coded
half-way bounce-back."""

import numpy as np
import pytest

from oracle import lattices as L
from oracle import lbm as O
from paper_1712_08288_gb300 import workloads as W

RHO0 = 1.0
RULES = {  # Sec. 3: l = gamma, 1.5 gamma, 2 gamma, gamma^2, gamma^2 + gamma  as (c0, c1, c2)
    "g": (0, 1, 0), "1.5g": (0, 1.5, 0), "2g": (0, 2, 0), "g2": (0, 0, 1), "g2+g": (0, 1, 1)}


def _coeffs(gamma, l, b=1.0):
    """Read the linear coefficients of the oracle's boundary_value off unit inputs."""
    w, e = 1 / 9, np.array([1, 0, 0])
    z = np.zeros(3)
    basis = np.eye(4)
    out = [O.boundary_value(w, e, gamma, l, b, RHO0, z, *basis[k]) for k in range(4)]
    wall = O.boundary_value(w, e, gamma, l, b, RHO0, np.array([1.0, 0, 0]), 0, 0, 0, 0)
    return np.array(out), wall


@pytest.mark.parametrize("gamma", [0.05, 0.25, 0.5, 0.75, 1.0])
@pytest.mark.parametrize("rule", list(RULES))
def test_single_node_closed_form(gamma, rule):
    """Eq. (2.10): coefficients (1+l-2g)/(1+l) on f_ibar(t), l/(1+l) on f'_i,
    (2g-l)/(1+l) on f'_ibar, 2/(1+l) w rho0 e.phi/c_s^2 for the wall, nothing on
    f_i(t) when b = 1; they are convex (Eq. (2.12)) and sum to one."""
    l = O.l_of_gamma(gamma, *RULES[rule])
    (c_fi, c_fib, c_pi, c_pib), wall = _coeffs(gamma, l)
    assert c_fi == 0.0
    assert abs(c_fib - (1 + l - 2 * gamma) / (1 + l)) < 1e-15
    assert abs(c_pi - l / (1 + l)) < 1e-15
    assert abs(c_pib - (2 * gamma - l) / (1 + l)) < 1e-15
    assert abs(wall - 2 / (1 + l) * (1 / 9) * RHO0 * 1.0 * 3) < 1e-15
    assert abs(c_fib + c_pi + c_pib - 1) < 1e-15
    assert O.is_convex(gamma, l)
    assert min(c_fib, c_pi, c_pib) >= -1e-15


@pytest.mark.parametrize("b", [0.2, 0.7, 1.0])
def test_b_combination(b):
    """Eq. (2.13): (1 - b) f_i(t) + b * (Eq. (2.10))."""
    gamma, l = 0.3, 0.45
    c1, w1 = _coeffs(gamma, l, 1.0)
    cb, wb = _coeffs(gamma, l, b)
    assert abs(cb[0] - (1 - b)) < 1e-15
    assert np.abs(cb[1:] - b * c1[1:]).max() < 1e-15
    assert abs(wb - b * w1) < 1e-15


def test_gspk_special_case():
    """Remark (4): l = gamma gives the single-node scheme of Geier et al. (2015):
    (1-g)/(1+g) f_ibar(t) + g/(1+g) [f'_i + f'_ibar] + 2/(1+g) w rho0 e.phi/c_s^2."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        g = rng.uniform(0.01, 1.0)
        fi, fib, pi, pib = rng.uniform(0, 0.2, 4)
        phi = 0.05 * rng.standard_normal(3)
        e = np.array([1, -1, 0])
        w = 1 / 36
        got = O.boundary_value(w, e, g, g, 1.0, RHO0, phi, fi, fib, pi, pib)
        want = ((1 - g) / (1 + g) * fib + g / (1 + g) * (pi + pib)
                + 2 / (1 + g) * w * RHO0 * (e @ phi) * 3)
        assert abs(got - want) < 1e-15


def test_zy2017_l0_special_case():
    """Remark (5): l = 0 gives (1-2g) f_ibar(t) + 2g f'_ibar + 2 w rho0 e.phi/c_s^2
    (non-convex for g > 1/2, Eq. (2.12))."""
    g = 0.3
    (c_fi, c_fib, c_pi, c_pib), wall = _coeffs(g, 0.0)
    assert (c_fi, c_pi) == (0.0, 0.0)
    assert abs(c_fib - (1 - 2 * g)) < 1e-15 and abs(c_pib - 2 * g) < 1e-15
    assert not O.is_convex(0.75, 0.0)


def test_half_way_value_is_bounce_back():
    """gamma = 1/2, l = 0, b = 1 is the half-way bounce-back rule (2.6) applied at x_f:
    f_i(x_f, t+1) = f'_ibar(x_f, t) + 2 w rho0 e_i.phi / c_s^2."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        fi, fib, pi, pib = rng.uniform(0, 0.2, 4)
        phi = 0.05 * rng.standard_normal(3)
        e = np.array([0, 1, 0])
        got = O.boundary_value(1 / 9, e, 0.5, 0.0, 1.0, RHO0, phi, fi, fib, pi, pib)
        assert got == pib + 2 * (1 / 9) * RHO0 * (e @ phi) / (1 / 3)


def _hwbb_channel_step(lat, f, S, g, nx, ny, solid, uw_row):
    """Separately coded LBM step with textbook half-way bounce-back (Ladd 1994) on a
    channel whose solid rows are given: pure Python loops over nodes and directions."""
    fp = np.full_like(f, np.nan)
    fl = ~solid
    fp[:, fl] = O.collide(lat, f[:, fl], S, RHO0, g)
    out = np.full_like(f, np.nan)
    for y in range(ny):
        for x in range(nx):
            n = x + nx * y
            if solid[n]:
                continue
            for i in range(lat.Q):
                xs, ys = (x - lat.e[i, 0]) % nx, (y - lat.e[i, 1]) % ny
                src = xs + nx * ys
                if not solid[src]:
                    out[i, n] = fp[i, src]
                else:   # the population arrives bounced back from the wall
                    ib = lat.opp[i]
                    out[i, n] = fp[ib, n] + 2 * lat.w[i] * RHO0 * (lat.e[i] @ uw_row[ys]) * 3
    return out


def test_channel_with_half_way_walls_equals_bounce_back():
    """A whole simulation: channel with walls exactly half-way (gamma = 1/2), moving top
    wall, body force, l = 0, b = 1 equals the bounce-back simulation bitwise-close."""
    lat = L.D2Q9
    nx, Ny = 4, 7
    w = W.poiseuille_2d(Ny, 0.5, 1.2, nx=nx)
    ny = Ny + 1
    uw_row = np.zeros((ny, 3))
    uw_row[Ny] = [0.01, 0, 0]            # top wall moves along x
    links = dict(w["links"])
    yb = (links["node"] // nx) + lat.e[links["d"], 1]
    links["uw"] = uw_row[yb]
    S = W.relaxation_rates("D2Q9", 1.2)
    g = np.array([1e-5, 0, 0])
    sim = O.Simulation(lat, w["shape"], S, RHO0, w["solid"], links, scheme=(0, 0, 0, 1.0), force=g)
    sim.init_equilibrium()
    f = sim.f.copy()
    for _ in range(20):
        sim.step()
        f = _hwbb_channel_step(lat, f, S, g, nx, ny, w["solid"], uw_row)
        assert np.abs(sim.f[:, ~w["solid"]] - f[:, ~w["solid"]]).max() < 1e-16


@pytest.mark.parametrize("rule", list(RULES))
@pytest.mark.parametrize("b", [1.0, 0.6])
def test_rest_state_is_fixed_point_with_curved_walls(rule, b):
    """f = w rho0 with phi = 0 stays put for any gamma, l and b (Eqs. (2.10), (2.13):
    the coefficients sum to one and the wall term vanishes)."""
    wk = W.couette_2d(24, (12.3, 11.6), 3.1, 10.2, 0.0)
    sim = O.Simulation(L.D2Q9, wk["shape"], W.relaxation_rates("D2Q9", 1.3), RHO0,
                       wk["solid"], wk["links"], scheme=RULES[rule] + (b,))
    sim.init_equilibrium()
    f0 = sim.f.copy()
    sim.step(5)
    fl = ~wk["solid"]
    assert np.abs(sim.f[:, fl] - f0[:, fl]).max() < 1e-15


def test_half_way_closed_channel_conserves_mass():
    """With half-way walls at rest (gamma = 1/2, l = 0) bounce-back returns every
    population to the fluid: total mass is conserved exactly, whatever the state."""
    nx, Ny = 5, 8
    w = W.poiseuille_2d(Ny, 0.5, 1.0, nx=nx)
    sim = O.Simulation(L.D2Q9, w["shape"], W.relaxation_rates("D2Q9", 1.0), RHO0,
                       w["solid"], w["links"], scheme=(0, 0, 0, 1.0))
    rho, u = W.random_state(w["shape"], "D2Q9", RHO0, 0.01, 3)
    sim.init_equilibrium(rho, u)
    m0 = sim.mass()
    sim.step(30)
    assert abs(sim.mass() - m0) < 1e-13 * m0


def test_two_node_yms2003_special_case():
    """Remark (4): with l = gamma the two-node scheme (Eq. 2.11) is the scheme of Yu,
    Mei & Shyy (2003): (1-g)/(1+g) f'_ibar(x_l) + g/(1+g) [f'_i + f'_ibar] +
    2/(1+g) w rho0 e.phi/c_s^2 -- the exact f_ibar(x_f, t+1) = f'_ibar(x_l, t) takes
    the place of Eq. (2.9)'s f_ibar(x_f, t)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        g = rng.uniform(0.01, 1.0)
        fi, fib, pi, pib, pl = rng.uniform(0, 0.2, 5)
        phi = 0.05 * rng.standard_normal(3)
        e = np.array([0, 1, -1])
        w = 1 / 36
        got = O.boundary_value(w, e, g, g, 1.0, RHO0, phi, fi, fib, pi, pib, f_ibar_next=pl)
        want = ((1 - g) / (1 + g) * pl + g / (1 + g) * (pi + pib)
                + 2 / (1 + g) * w * RHO0 * (e @ phi) * 3)
        assert abs(got - want) < 1e-15


def test_two_node_equals_single_node_for_halfway_bounce_back():
    """gamma = 1/2, l = 0: the weight of f_ibar(x_f, t+1) is (1 + l - 2 gamma)/(1 + l)
    = 0, so both schemes give half-way bounce-back whatever x_l holds."""
    rng = np.random.default_rng(2)
    fi, fib, pi, pib, pl = rng.uniform(0, 0.2, 5)
    phi = np.array([0.01, -0.02, 0.0])
    e = np.array([1, 0, 0])
    a = O.boundary_value(1 / 9, e, 0.5, 0.0, 1.0, RHO0, phi, fi, fib, pi, pib)
    b = O.boundary_value(1 / 9, e, 0.5, 0.0, 1.0, RHO0, phi, fi, fib, pi, pib, f_ibar_next=pl)
    assert a == b
