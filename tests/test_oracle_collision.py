"""Pins of the oracle's equilibrium and MRT collision (Appendix of arXiv:1712.08288)
against closed forms from the literature and textbook special cases."""

import numpy as np
import pytest

from oracle import lattices as L
from oracle import lbm as O

RHO0 = 1.0


def _random_f(lat, n, seed, scale=0.05):
    rng = np.random.default_rng(seed)
    return lat.w[:, None] * (1.0 + scale * rng.standard_normal((lat.Q, n)))


def test_d3q15_equilibrium_moments_dhumieres():
    """M f^eq for the Appendix's D3Q15 equals the D3Q15 equilibrium moments of
    d'Humieres et al. (2002) in incompressible form (j/rho0): e = -rho + j^2/rho0,
    eps = rho - 5 j^2/rho0, q = -7/3 j, 3p_xx = (3jx^2 - j^2)/rho0,
    p_ww = (jy^2 - jz^2)/rho0, p_ab = ja jb/rho0, m_xyz = 0."""
    rng = np.random.default_rng(4)
    n = 40
    rho = 1 + 0.1 * rng.standard_normal(n)
    u = 0.05 * rng.standard_normal((3, n))
    jx, jy, jz = RHO0 * u
    j2 = jx * jx + jy * jy + jz * jz
    z = np.zeros(n)
    want = np.array([rho, -rho + j2 / RHO0, rho - 5 * j2 / RHO0,
                     jx, -7 / 3 * jx, jy, -7 / 3 * jy, jz, -7 / 3 * jz,
                     (3 * jx * jx - j2) / RHO0, (jy * jy - jz * jz) / RHO0,
                     jx * jy / RHO0, jy * jz / RHO0, jx * jz / RHO0, z])
    got = L.D3Q15.M @ O.equilibrium(L.D3Q15, rho, u, RHO0)
    assert np.abs(got - want).max() < 1e-14


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q15, L.D3Q19])
def test_equilibrium_moments_closed_form(lat):
    """Incompressible equilibrium (He & Luo 1997; Eq. (42)): sum f^eq = rho,
    sum c f^eq = rho0 u, sum c c f^eq = rho c_s^2 I + rho0 u u."""
    rng = np.random.default_rng(1)
    n = 50
    rho = 1 + 0.1 * rng.standard_normal(n)
    u = np.zeros((3, n))
    u[: lat.D] = 0.05 * rng.standard_normal((lat.D, n))
    feq = O.equilibrium(lat, rho, u, RHO0)
    e = lat.e.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-15)
    assert np.allclose(e.T @ feq, RHO0 * u, rtol=0, atol=1e-15)
    P = np.einsum("ia,ib,in->abn", e, e, feq)
    want = rho[None, None, :] / 3 * np.eye(3)[:, :, None] + RHO0 * np.einsum("an,bn->abn", u, u)
    D = lat.D
    assert np.abs(P[:D, :D] - want[:D, :D]).max() < 1e-15


def test_d2q9_equilibrium_moments_lallemand_luo():
    """M f^eq for D2Q9 equals the incompressible equilibrium moments of Lallemand &
    Luo (2000): e = -2 rho + 3 j^2/rho0, eps = rho - 3 j^2/rho0, q = -j,
    p_xx = (jx^2 - jy^2)/rho0, p_xy = jx jy/rho0."""
    rng = np.random.default_rng(2)
    n = 40
    rho = 1 + 0.1 * rng.standard_normal(n)
    u = np.zeros((3, n))
    u[:2] = 0.05 * rng.standard_normal((2, n))
    jx, jy = RHO0 * u[0], RHO0 * u[1]
    j2 = jx * jx + jy * jy
    want = np.array([rho, -2 * rho + 3 * j2 / RHO0, rho - 3 * j2 / RHO0, jx, -jx, jy, -jy,
                     (jx * jx - jy * jy) / RHO0, jx * jy / RHO0])
    got = L.D2Q9.M @ O.equilibrium(L.D2Q9, rho, u, RHO0)
    assert np.abs(got - want).max() < 1e-14


def test_d3q19_equilibrium_moments_dhumieres():
    """M f^eq for D3Q19 equals the equilibrium moments of d'Humieres et al. (2002)
    with w_eps = 3, w_epsj = -11/2, w_xx = -1/2 (incompressible form, j/rho0):
    e = -11 rho + 19 j^2/rho0, eps = 3 rho - 11/2 j^2/rho0, q = -2/3 j,
    3p_xx = (3jx^2 - j^2)/rho0, 3pi_xx = -1/2 3p_xx, p_ww = (jy^2 - jz^2)/rho0,
    pi_ww = -1/2 p_ww, p_ab = ja jb/rho0, m = 0."""
    rng = np.random.default_rng(3)
    n = 40
    rho = 1 + 0.1 * rng.standard_normal(n)
    u = 0.05 * rng.standard_normal((3, n))
    jx, jy, jz = RHO0 * u
    j2 = jx * jx + jy * jy + jz * jz
    pxx = (3 * jx * jx - j2) / RHO0
    pww = (jy * jy - jz * jz) / RHO0
    z = np.zeros(n)
    want = np.array([rho, -11 * rho + 19 * j2 / RHO0, 3 * rho - 5.5 * j2 / RHO0,
                     jx, -2 / 3 * jx, jy, -2 / 3 * jy, jz, -2 / 3 * jz,
                     pxx, -0.5 * pxx, pww, -0.5 * pww,
                     jx * jy / RHO0, jy * jz / RHO0, jx * jz / RHO0, z, z, z])
    got = L.D3Q19.M @ O.equilibrium(L.D3Q19, rho, u, RHO0)
    assert np.abs(got - want).max() < 1e-14


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q15, L.D3Q19])
def test_equal_rates_reduce_to_bgk(lat):
    """S = s I turns the MRT operator into the BGK operator f' = f - s (f - f^eq)."""
    f = _random_f(lat, 30, 4)
    s = 1.37
    rho = f.sum(0)
    u = lat.e.T.astype(float) @ f / RHO0
    bgk = f - s * (f - O.equilibrium(lat, rho, u, RHO0))
    got = O.collide(lat, f, np.full(lat.Q, s), RHO0, np.zeros(3))
    assert np.abs(got - bgk).max() < 1e-15


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q15, L.D3Q19])
def test_collision_invariants_and_moment_relaxation(lat):
    """rho is invariant, j gains exactly rho0 g, and every other moment relaxes on
    its own: m'_k = m_k - s_k (m_k - m^eq_k) (the meaning of a diagonal S)."""
    rng = np.random.default_rng(5)
    f = _random_f(lat, 30, 6)
    S = rng.uniform(0.3, 1.9, lat.Q)
    g = np.array([1e-3, -2e-3, 5e-4])
    fp = O.collide(lat, f, S, RHO0, g)
    rho, j = O.density_momentum(lat, f)
    rho2, j2 = O.density_momentum(lat, fp)
    assert np.abs(rho2 - rho).max() < 1e-15
    assert np.abs(j2[: lat.D] - (j[: lat.D] + RHO0 * g[: lat.D, None])).max() < 1e-15
    m = lat.M @ f
    meq = lat.M @ O.equilibrium(lat, rho, j / RHO0, RHO0)
    mp = lat.M @ fp
    others = [k for k in range(lat.Q) if k != 0 and k not in lat.j_rows]
    want = m[others] - S[others, None] * (m[others] - meq[others])
    assert np.abs(mp[others] - want).max() < 1e-13


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19])
def test_uniform_equilibrium_is_fixed_point(lat):
    """A uniform f^eq(rho0, u0) in a fully periodic box is a fixed point of
    collision + advection (no force)."""
    shape = (5, 4, 1 if lat.D == 2 else 3)
    N = shape[0] * shape[1] * shape[2]
    sim = O.Simulation(lat, shape, np.linspace(0.6, 1.8, lat.Q), RHO0, np.zeros(N, bool),
                       dict(node=[], d=[], q=[], uw=np.zeros((0, 3))))
    u0 = np.tile([0.03, -0.02, 0.01 if lat.D == 3 else 0.0], (N, 1))
    sim.init_equilibrium(np.full(N, 1.02), u0)
    f0 = sim.f.copy()
    sim.step(3)
    assert np.abs(sim.f - f0).max() < 1e-15


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19])
def test_periodic_mass_and_momentum_conservation(lat):
    """Fully periodic box, random state: total mass is conserved and total momentum
    grows by exactly rho0 g per node per step."""
    shape = (6, 5, 1 if lat.D == 2 else 4)
    N = shape[0] * shape[1] * shape[2]
    g = np.array([2e-4, -1e-4, 3e-4 if lat.D == 3 else 0.0])
    sim = O.Simulation(lat, shape, np.linspace(0.6, 1.8, lat.Q), RHO0, np.zeros(N, bool),
                       dict(node=[], d=[], q=[], uw=np.zeros((0, 3))), force=g, skew=(0, 0))
    sim.f = _random_f(lat, N, 7)
    m0 = sim.f.sum()
    j0 = (lat.e.T.astype(float) @ sim.f).sum(1)
    sim.step(4)
    assert abs(sim.f.sum() - m0) < 1e-12
    j1 = (lat.e.T.astype(float) @ sim.f).sum(1)
    assert np.abs(j1 - (j0 + 4 * N * RHO0 * g)).max() < 1e-12


def test_translation_equivariance_with_skew():
    """Translating the initial state of a skew-periodic box by one node in x translates
    the result exactly (the skewed wrap is a symmetry of the discrete problem)."""
    lat = L.D3Q19
    shape, skew = (6, 4, 4), (1, 3)
    N = 6 * 4 * 4
    mk = lambda: O.Simulation(lat, shape, np.linspace(0.6, 1.8, lat.Q), RHO0, np.zeros(N, bool),
                              dict(node=[], d=[], q=[], uw=np.zeros((0, 3))), skew=skew)
    a, b = mk(), mk()
    a.f = _random_f(lat, N, 8)
    # b's node x holds a's node x - 1 (with the skewed wrap)
    x = np.arange(N) % 6
    y = (np.arange(N) // 6) % 4
    z = np.arange(N) // 24
    src = O.wrapped_index(shape, skew, x - 1, y, z)
    b.f = a.f[:, src]
    a.step(3)
    b.step(3)
    assert np.array_equal(b.f, a.f[:, src])


def test_wrapped_index_skew():
    shape, skew = (8, 5, 7), (2, 3)
    # one x-period back is the translation (nx, sy, sz)
    assert O.wrapped_index(shape, skew, 8 + 1, 2 + 2, 3 + 3) == 1 + 8 * (2 + 5 * 3)
    assert O.wrapped_index(shape, skew, -1, 0, 0) == 7 + 8 * ((0 + 2) % 5 + 5 * ((0 + 3) % 7))
