"""The input generators: wall fractions against bisection on the exact surfaces,
cut-link completeness, seeded reproducibility."""

import numpy as np

from paper_1712_08288_gb300 import workloads as W


def _bisect(inside_solid, p, d, lo=0.0, hi=1.0, it=80):
    """First crossing of the wall along p + t d, t in (0, 1] (p fluid, p + d solid)."""
    for _ in range(it):
        mid = 0.5 * (lo + hi)
        if inside_solid(p + mid * d):
            hi = mid
        else:
            lo = mid
    return hi


def test_couette_fractions_by_bisection():
    w = W.couette_2d(40, (20.3, 19.6), 6.2, 17.5, 0.01)
    E = W.DIRECTIONS["D2Q9"].astype(float)
    c = np.array([20.3, 19.6, 0.0])

    def solid(p):
        r = np.hypot(p[0] - c[0], p[1] - c[1])
        return not (6.2 < r < 17.5)
    L = w["links"]
    nx = 40
    for k in range(0, len(L["node"]), 7):
        n = L["node"][k]
        p = np.array([n % nx, n // nx, 0.0])
        q = _bisect(solid, p, E[L["d"][k]])
        assert abs(q - L["q"][k]) < 1e-12


def test_couette_wall_velocity_is_tangential():
    U1, R1 = 0.02, 6.2
    w = W.couette_2d(40, (20.3, 19.6), R1, 17.5, U1)
    L = w["links"]
    E = W.DIRECTIONS["D2Q9"].astype(float)
    nx = 40
    for k in range(len(L["node"])):
        n = L["node"][k]
        xb = np.array([n % nx, n // nx, 0.0]) + L["q"][k] * E[L["d"][k]] - [20.3, 19.6, 0]
        uw = L["uw"][k]
        if np.hypot(*xb[:2]) < 10:          # inner wall
            assert abs(np.hypot(*xb[:2]) - R1) < 1e-9
            assert abs(np.linalg.norm(uw) - U1) < 1e-12
            assert abs(uw @ xb) < 1e-12     # tangential
            assert xb[0] * uw[1] - xb[1] * uw[0] > 0  # counter-clockwise
        else:
            assert not uw.any()


def test_pipe_fractions_by_bisection():
    w = W.tilted_pipe_3d(32)
    a, R = w["axis"], w["radius"]
    E = W.DIRECTIONS["D3Q19"].astype(float)
    c0 = np.array([16, 16 + 0.37, 16 + 0.21])
    ims = [np.array([0, my * 32, mz * 32.0]) for my in (-1, 0, 1) for mz in (-1, 0, 1)]

    def dist(p):
        best = np.inf
        for im in ims:
            v = p - c0 - im
            v = v - (v @ a) * a
            best = min(best, np.linalg.norm(v))
        return best
    L = w["links"]
    for k in range(0, len(L["node"]), 37):
        n = L["node"][k]
        p = np.array([n % 32, (n // 32) % 32, n // 1024], dtype=float)
        q = _bisect(lambda x: dist(x) >= R, p, E[L["d"][k]])
        assert abs(q - L["q"][k]) < 1e-10


def test_links_complete_and_sorted():
    w = W.tilted_pipe_3d(16)
    node, d = W.cut_links("D3Q19", w["shape"], w["skew"], w["solid"])
    assert np.array_equal(node, w["links"]["node"]) and np.array_equal(d, w["links"]["d"])
    assert np.all(np.diff(node) >= 0)
    assert not w["solid"][node].any()
    assert np.all((w["links"]["q"] > 0) & (w["links"]["q"] <= 1))


def test_ensemble_is_seeded():
    a = W.couette_ensemble(96, 0)
    b = W.couette_ensemble(96, 0)
    assert a == b
    assert all(48 <= p["n"] <= 768 for p in a)
    assert all(0.1 * p["n"] <= p["R1"] <= 0.25 * p["n"] for p in a)


def test_trt_rows_follow_the_parity_of_m():
    """The TRT vector puts s_minus exactly on the rows of M that are odd under
    e -> -e (checked against the oracle's matrices) and satisfies the magic product."""
    import numpy as np
    from oracle import lattices as OL
    for name in ("D2Q9", "D3Q19", "D3Q15"):
        lat = OL.BY_NAME[name]
        s = W.relaxation_rates_trt(name, 1.3, magic=0.25)
        odd = np.array([np.allclose(lat.M[k][lat.opp], -lat.M[k]) for k in range(lat.Q)])
        sm = s[odd]
        assert np.allclose(sm, sm[0]) and np.allclose(s[~odd], 1.3)
        assert abs((1 / 1.3 - 0.5) * (1 / sm[0] - 0.5) - 0.25) < 1e-14
        assert np.all(W.relaxation_rates_bgk(name, 0.9) == 0.9)


def test_taylor_green_disc_generator():
    """Sec. 3.2 inputs: every cut link's wall point lies on the circle of radius 1/4
    about (1/2, 1/2), q in (0, 1], nodes on the rim are solid, the wall velocity is
    the analytic field at the wall point (in lattice units), and T = 1/U0 in steps."""
    import numpy as np
    inv_h, s_nu = 40, 1.0
    w = W.taylor_green_disc(inv_h, s_nu)
    h = 1.0 / inv_h
    n = inv_h + 1
    node, d, q, uw = (w["links"][k] for k in ("node", "d", "q", "uw"))
    E = W.DIRECTIONS["D2Q9"]
    x, y = (node % n) * h, (node // n) * h
    xb, yb = x + q * E[d, 0] * h, y + q * E[d, 1] * h
    assert np.allclose(np.hypot(xb - 0.5, yb - 0.5), 0.25, atol=1e-12, rtol=0)
    assert np.all((q > 0) & (q <= 1))
    X, Y = (np.arange(n * n) % n) * h, (np.arange(n * n) // n) * h
    on_rim = np.isclose(np.hypot(X - 0.5, Y - 0.5), 0.25, atol=1e-12)
    assert on_rim.any() and np.all(w["solid"][on_rim])
    eta = (1 / s_nu - 0.5) / (3 * 0.002)
    u_b = -0.05 * np.cos(2 * np.pi * xb) * np.sin(2 * np.pi * yb) * eta * h
    v_b = 0.05 * np.cos(2 * np.pi * yb) * np.sin(2 * np.pi * xb) * eta * h
    assert np.allclose(uw[:, 0], u_b, atol=1e-15) and np.allclose(uw[:, 1], v_b, atol=1e-15)
    assert abs(w["steps"] * eta * h * h - 1 / 0.05) < eta * h * h
    assert abs(w["decay"] - np.exp(-8 * np.pi ** 2 * 0.002 * eta * h * h)) < 1e-15
