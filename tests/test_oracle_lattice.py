"""Pins of the oracle's lattice tables against what the paper prints and what the
mathematics of the lattices fixes (Appendix of arXiv:1712.08288)."""

import os

import numpy as np
import pytest

from oracle import lattices as L
from paper_1712_08288_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_matrix(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def _load_constants():
    out = {}
    with open(os.path.join(GOLDEN, "lattice_constants.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                lat, qty, *vals = line.split()
                out[(lat, qty)] = np.array([float(v) for v in vals])
    return out


def test_printed_matrices_match():
    """Appendix, eqn:matrix-m and eqn:matrix-m3, entry by entry."""
    assert np.array_equal(L.D2Q9.M, _load_matrix("d2q9_matrix_m.txt"))
    assert np.array_equal(L.D3Q15.M, _load_matrix("d3q15_matrix_m.txt"))


def test_printed_velocities_and_weights():
    c = _load_constants()
    for lat, scale in ((L.D2Q9, 36), (L.D3Q15, 72)):
        for k, ax in enumerate("xyz"[: 3 if lat.D == 3 else 2]):
            assert np.array_equal(lat.e[:, k], c[(lat.name, "e" + ax)])
        assert np.allclose(lat.w * scale, c[(lat.name, "w%d" % scale)], rtol=0, atol=1e-13)


def test_d2q9_matches_lallemand_luo_polynomials():
    """The printed D2Q9 table equals the Lallemand-Luo (2000) polynomial moments
    1, 3|e|^2-4, (9|e|^4-21|e|^2+8)/2, e_x, (3|e|^2-5)e_x, e_y, (3|e|^2-5)e_y,
    e_x^2-e_y^2, e_x e_y, evaluated on the Appendix velocities."""
    e = L.D2Q9.e.astype(float)
    x, y = e[:, 0], e[:, 1]
    r2 = x * x + y * y
    rows = [np.ones(9), 3 * r2 - 4, (9 * r2 * r2 - 21 * r2 + 8) / 2, x, (3 * r2 - 5) * x,
            y, (3 * r2 - 5) * y, x * x - y * y, x * y]
    assert np.array_equal(np.array(rows), L.D2Q9.M)


@pytest.mark.parametrize("lat,norms", [
    (L.D2Q9, [9, 36, 36, 6, 12, 6, 12, 4, 4]),
    (L.D3Q15, [15, 18, 360, 10, 40, 10, 40, 10, 40, 12, 4, 8, 8, 8, 8]),
    (L.D3Q19, [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]),
])
def test_rows_orthogonal_with_known_norms(lat, norms):
    G = lat.M @ lat.M.T
    assert np.array_equal(G, np.diag(np.array(norms, dtype=float)))


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q15, L.D3Q19])
def test_inverse(lat):
    assert np.abs(lat.M @ lat.Minv - np.eye(lat.Q)).max() < 1e-14
    assert np.abs(lat.Minv @ lat.M - np.eye(lat.Q)).max() < 1e-14


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q15, L.D3Q19])
def test_weight_isotropy(lat):
    """sum w = 1, sum w e = 0, sum w e e = c_s^2 I, sum w e e e e = c_s^4 (dd+dd+dd)."""
    e = lat.e.astype(float)[:, : lat.D]
    w = lat.w
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ e).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, e, e) - np.eye(lat.D) / 3).max() < 1e-15
    T4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    I = np.eye(lat.D)
    want = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
            + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.abs(T4 - want).max() < 1e-15


def test_opposites():
    assert list(L.D2Q9.opp) == [0, 3, 4, 1, 2, 7, 8, 5, 6]
    assert list(L.D3Q15.opp) == [0, 2, 1, 4, 3, 6, 5, 14, 13, 12, 11, 10, 9, 8, 7]
    assert list(L.D3Q19.opp) == [0] + [k + 1 if k % 2 else k - 1 for k in range(1, 19)]


def test_api_direction_numbering_agrees():
    """The oracle's velocity order is the C-ABI's numbering used by the input generators."""
    assert np.array_equal(L.D2Q9.e, W.DIRECTIONS["D2Q9"])
    assert np.array_equal(L.D3Q19.e, W.DIRECTIONS["D3Q19"])
