"""Lattice definitions for the oracle (test infrastructure only, see package docstring).

Sources
-------
* D2Q9: velocities, weights and sound speed from the Appendix (D2Q9 paragraph);
  transformation matrix M exactly as printed in the Appendix (matrix labelled
  eqn:matrix-m, Lallemand & Luo 2000 row order rho, e, eps, j_x, q_x, j_y, q_y,
  p_xx, p_xy).
* D3Q15: velocities, weights and M exactly as printed in the Appendix (matrix
  labelled eqn:matrix-m3).
* D3Q19: not in the paper.  The Appendix cites d'Humieres et al. (2002) for the 3D
  MRT models; the D3Q19 model of that reference is used here: rest, the six face
  neighbours and the twelve edge neighbours, weights 1/3, 1/18, 1/36, and the
  nineteen orthogonal polynomial moments of that reference.  The direction order is
  the one the C-ABI declares (rest; +x,-x,+y,-y,+z,-z; then the twelve edges with
  each direction followed by its opposite).

All lattices are in lattice units (h = delta_t = c = 1) with c_s^2 = 1/3
(Appendix: c_s = c/sqrt(3) for all three models).

The inverse of M is taken from a generic dense inverse (numpy.linalg.inv), not
from the orthogonality of the rows, so that the identity M M^-1 = I is a check of
the printed tables rather than an assumption.
"""

from dataclasses import dataclass, field

import numpy as np

CS2 = 1.0 / 3.0  # c_s^2 in lattice units (Appendix)


@dataclass
class Lattice:
    name: str
    D: int                      # spatial dimension
    e: np.ndarray               # (Q, 3) integer velocities (third column 0 in 2D)
    w: np.ndarray               # (Q,) weights omega_i
    M: np.ndarray               # (Q, Q) transformation matrix, float64
    j_rows: tuple               # rows of M that are the momentum components j_x, j_y(, j_z)
    opp: np.ndarray = field(init=False)
    Minv: np.ndarray = field(init=False)

    @property
    def Q(self):
        return self.e.shape[0]

    def __post_init__(self):
        # opposite index: e_{opp(i)} = -e_i (Sec. 2, text after Eq. (2.6))
        opp = np.empty(self.Q, dtype=np.int64)
        for i in range(self.Q):
            matches = [k for k in range(self.Q) if np.all(self.e[k] == -self.e[i])]
            assert len(matches) == 1
            opp[i] = matches[0]
        self.opp = opp
        self.Minv = np.linalg.inv(self.M)


def _d2q9():
    # Appendix, D2Q9: columns i = 0..8 of (e_ix, e_iy)
    ex = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    ey = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    e = np.array([[a, b, 0] for a, b in zip(ex, ey)], dtype=np.int64)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    # Appendix, matrix eqn:matrix-m, as printed
    M = np.array([
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1],
    ], dtype=np.float64)
    return Lattice("D2Q9", 2, e, w, M, (3, 5))


def _d3q15():
    # Appendix, D3Q15 velocities
    ex = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1]
    ey = [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]
    ez = [0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1]
    e = np.array(list(zip(ex, ey, ez)), dtype=np.int64)
    w = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)
    # Appendix, matrix eqn:matrix-m3, as printed
    M = np.array([
        [1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-2, -1, -1, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1],
        [16, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1],
        [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1],
        [0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1],
        [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1],
        [0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1],
        [0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1],
        [0, 0, 0, 0, 0, -4, 4, 1, 1, 1, 1, -1, -1, -1, -1],
        [0, 2, 2, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1],
        [0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1],
        [0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1],
        [0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1],
    ], dtype=np.float64)
    return Lattice("D3Q15", 3, e, w, M, (3, 5, 7))


def _d3q19():
    # direction order of the C-ABI: rest, faces (+x,-x,+y,-y,+z,-z), edges in
    # opposite pairs
    e = np.array([
        (0, 0, 0),
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
    ], dtype=np.int64)
    r2 = (e * e).sum(1)
    w = np.where(r2 == 0, 1 / 3, np.where(r2 == 1, 1 / 18, 1 / 36))
    x, y, z = (e[:, k].astype(np.float64) for k in range(3))
    r2 = r2.astype(np.float64)
    # d'Humieres, Ginzburg, Krafczyk, Lallemand & Luo (2002), D3Q19 moment basis:
    # rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww, pi_ww,
    # p_xy, p_yz, p_xz, m_x, m_y, m_z
    rows = [
        np.ones_like(r2),
        19 * r2 - 30,
        (21 * r2 * r2 - 53 * r2 + 24) / 2,
        x, (5 * r2 - 9) * x,
        y, (5 * r2 - 9) * y,
        z, (5 * r2 - 9) * z,
        3 * x * x - r2, (3 * r2 - 5) * (3 * x * x - r2),
        y * y - z * z, (3 * r2 - 5) * (y * y - z * z),
        x * y, y * z, x * z,
        (y * y - z * z) * x, (z * z - x * x) * y, (x * x - y * y) * z,
    ]
    M = np.array(rows, dtype=np.float64)
    return Lattice("D3Q19", 3, e, w, M, (3, 5, 7))


D2Q9 = _d2q9()
D3Q15 = _d3q15()
D3Q19 = _d3q19()

BY_NAME = {lat.name: lat for lat in (D2Q9, D3Q15, D3Q19)}

