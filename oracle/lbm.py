"""One lattice-Boltzmann time step with the paper's boundary schemes, in plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written from Zhao & Yong,
"A family of single-node second-order boundary schemes for the lattice Boltzmann
method" (arXiv:1712.08288):

* LBE and its split into collision and advection: Eqs. (2.1), (2.2a), (2.2b).
* MRT collision  Omega = -M^-1 S M (f - f^eq): Appendix.
* Incompressible equilibrium (He & Luo 1997): Appendix, Eq. (42); rho = sum f_i,
  rho0 u = sum c_i f_i (Appendix, text after Eq. (42)).
* Boundary: for a fluid node x_f whose neighbour x_r = x_f - e_i is outside the
  fluid, f_i(x_f, t+1) is built exactly in the paper's order: interpolation (2.5)
  toward x_1, half-way bounce-back (2.6) at x_1, interpolation (2.7) at x_2 with the
  approximation (2.9), and the b-combination (2.13).  l is a non-negative number per
  link (Sec. 2); here l = c0 + c1*gamma + c2*gamma^2 covers the five rules of Sec. 3
  (gamma, 1.5 gamma, 2 gamma, gamma^2, gamma^2 + gamma) and the l = 0 scheme.
* Relative L2 error E_r: Sec. 3.1, Eq. (eqn:L2-error).

Readings where the paper is silent (each one is listed in the design notes):

* Body force.  The paper drives its flows with a force F (Sec. 3) but states no
  forcing scheme.  Here rho0*g is added to the momentum moments after relaxation,
  in moment space only:  f' += M^-1 (0, .., rho0 g_alpha at the j_alpha rows, .., 0).
  The equilibrium uses u = j/rho0 of the pre-collision state, and the reported
  velocity is u = j/rho0 + g/2 (the mean of the pre- and post-force momentum).
* Lattice units throughout: h = delta_t = 1, c = 1, c_s^2 = 1/3, so the wall term
  of Eq. (2.6) is 2 w_i rho0 (e_i . phi) / c_s^2.
* The wall velocity phi(x_b) is given per cut link and held fixed in time.
* Periodicity: every axis wraps.  Optionally the x-wrap is skewed: the field is
  invariant under the translation (nx, sy, sz), which makes a pipe whose axis is
  parallel to (nx, sy, sz) periodic.  Walls that are not periodic are expressed
  by solid nodes.

Cut links are given in the C-ABI convention: (node, d, q, phi) with d the direction
that points from the fluid node x_f toward the wall, so that x_f + e_d is solid,
the population being computed is i = opp(d) (e_i = -e_d) and gamma = q
(x_b = x_f - gamma e_i, Sec. 2).
"""

import numpy as np

from .lattices import CS2


# ----------------------------------------------------------------------------
# grid and neighbours
# ----------------------------------------------------------------------------

def wrapped_index(shape, skew, X, Y, Z):
    """Linear index x + nx*(y + ny*z) of the periodic image of integer points.

    The field is invariant under (nx, sy, sz) and under (0, ny, 0), (0, 0, nz).
    """
    nx, ny, nz = shape
    sy, sz = skew
    X = np.asarray(X, dtype=np.int64)
    Y = np.asarray(Y, dtype=np.int64)
    Z = np.asarray(Z, dtype=np.int64)
    k = np.floor_divide(X, nx)          # how many x-periods the point lies away
    X = X - k * nx
    Y = np.mod(Y - k * sy, ny)
    Z = np.mod(Z - k * sz, nz)
    return X + nx * (Y + ny * Z)


def neighbour_table(lat, shape, skew):
    """nbr[i, n] = linear index of x_n + e_i (periodic image)."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    nbr = np.empty((lat.Q, nx * ny * nz), dtype=np.int64)
    for i in range(lat.Q):
        ex, ey, ez = lat.e[i]
        nbr[i] = wrapped_index(shape, skew, x + ex, y + ey, z + ez)
    return nbr


# ----------------------------------------------------------------------------
# equilibrium, moments, collision
# ----------------------------------------------------------------------------

def equilibrium(lat, rho, u, rho0):
    """Eq. (42): f_i^eq = w_i { rho + rho0 [ c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u^2/(2 c_s^2) ] }.

    rho: (N,), u: (3, N) (third row ignored in 2D).  Returns (Q, N).
    """
    c = lat.e.astype(np.float64)            # c_i = c e_i with c = 1
    cu = c @ u                              # (Q, N)
    u2 = (u * u).sum(axis=0)                # (N,)
    return lat.w[:, None] * (rho[None, :] + rho0 * (cu / CS2 + cu * cu / (2 * CS2 * CS2)
                                                   - u2[None, :] / (2 * CS2)))


def density_momentum(lat, f):
    """rho = sum_i f_i and rho0 u = sum_i c_i f_i (Appendix)."""
    rho = f.sum(axis=0)
    j = lat.e.T.astype(np.float64) @ f      # (3, N)
    return rho, j


def collide(lat, f, S, rho0, g):
    """Eq. (2.2a) with the MRT collision of the Appendix and the body-force reading.

    f' = f - M^-1 S M (f - f^eq) + M^-1 F_m, F_m = rho0 g at the momentum rows.
    """
    rho, j = density_momentum(lat, f)
    u = j / rho0
    feq = equilibrium(lat, rho, u, rho0)
    m_neq = lat.M @ (f - feq)
    fpost = f - lat.Minv @ (np.asarray(S, dtype=np.float64)[:, None] * m_neq)
    Fm = np.zeros(lat.Q)
    for a, row in enumerate(lat.j_rows):
        Fm[row] = rho0 * g[a]
    return fpost + (lat.Minv @ Fm)[:, None]


# ----------------------------------------------------------------------------
# the boundary scheme
# ----------------------------------------------------------------------------

def l_of_gamma(gamma, c0, c1, c2):
    """The family parameter l as a function of the wall fraction (Sec. 3 rules)."""
    return c0 + c1 * gamma + c2 * gamma * gamma


def is_convex(gamma, l):
    """Eq. (2.12): max{0, 2 gamma - 1} <= l <= 2 gamma."""
    return (l >= np.maximum(0.0, 2 * gamma - 1)) & (l <= 2 * gamma)


def boundary_value(w_i, e_i, gamma, l, b, rho0, phi,
                   f_i_t, f_ibar_t, fpost_i, fpost_ibar, f_ibar_next=None):
    """f_i(x_f, t+1) for one cut link, following Sec. 2 step by step.

    Inputs are the boundary node's own populations: f_i(x_f,t), f_ibar(x_f,t)
    (pre-collision) and f'_i(x_f,t), f'_ibar(x_f,t) (post-collision).  Every
    argument may also be an array over links (e_i and phi then have a last axis
    of length 3), in which case the formula is applied link by link.
    f_ibar_next: the two-node scheme (Remark (2) after Eq. 2.10, Eq. 2.11) passes
    the exact f_ibar(x_f, t+dt) = f'_ibar(x_l, t) of the fluid neighbour x_l here;
    None keeps the single-node approximation.
    """
    if f_ibar_next is None:
        # Eq. (2.9): f_ibar(x_f, t+dt) ~ f_ibar(x_f, t)
        f_ibar_next = f_ibar_t
    # Eq. (2.7): interpolation at x_2 between x_f (t+dt) and x_r, whose value at
    # t+dt is the advected f'_ibar(x_f, t)
    f_ibar_x2 = (1 + l - 2 * gamma) * f_ibar_next + (2 * gamma - l) * fpost_ibar
    # Eq. (2.6): half-way bounce-back across x_b, which lies midway between x_1, x_2
    e_dot_phi = (np.asarray(e_i) * np.asarray(phi)).sum(axis=-1)
    f_i_x1 = f_ibar_x2 + 2 * w_i * rho0 * e_dot_phi / CS2
    # Eq. (2.5): interpolation at x_f between x_l (advected f'_i(x_f,t)) and x_1
    rhs = l / (1 + l) * fpost_i + 1 / (1 + l) * f_i_x1
    # Eq. (2.13): convex combination with f_i(x_f, t)
    return (1 - b) * f_i_t + b * rhs


# ----------------------------------------------------------------------------
# simulation state
# ----------------------------------------------------------------------------

class Simulation:
    """Two-array LBM with push advection and the single-node boundary (2.13).

    shape = (nx, ny, nz) (nz = 1 in 2D); node index n = x + nx*(y + ny*z).
    solid: (N,) bool.  links: dict of arrays node, d, q (N_links,), uw (N_links, 3).
    scheme: (c0, c1, c2, b) for l = c0 + c1 q + c2 q^2 and the b of Eq. (2.13).
    """

    def __init__(self, lat, shape, S, rho0, solid, links, scheme=(0.0, 1.0, 0.0, 1.0),
                 force=(0.0, 0.0, 0.0), skew=(0, 0), two_node=False):
        self.lat = lat
        self.shape = tuple(int(s) for s in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.S = np.asarray(S, dtype=np.float64)
        assert self.S.shape == (lat.Q,)
        self.rho0 = float(rho0)
        self.solid = np.asarray(solid, dtype=bool).reshape(self.N)
        self.fluid = ~self.solid
        self.g = np.asarray(force, dtype=np.float64)
        self.skew = tuple(int(s) for s in skew)
        self.nbr = neighbour_table(lat, self.shape, self.skew)
        c0, c1, c2, b = scheme
        self.scheme_coeffs = (float(c0), float(c1), float(c2))
        self.b = float(b)
        assert 0.0 < self.b <= 1.0, "b must lie in (0, 1] (Eq. (2.13))"

        node = np.asarray(links["node"], dtype=np.int64)
        d = np.asarray(links["d"], dtype=np.int64)
        q = np.asarray(links["q"], dtype=np.float64)
        uw = np.asarray(links["uw"], dtype=np.float64).reshape(-1, 3) if len(node) else np.zeros((0, 3))
        # every fluid -> solid link must be listed exactly once, and nothing else
        want = set()
        for dd in range(lat.Q):
            for n in np.nonzero(self.fluid & self.solid[self.nbr[dd]])[0]:
                want.add((int(n), dd))
        got = set(zip(node.tolist(), d.tolist()))
        assert len(got) == len(node), "duplicate cut link"
        assert got == want, "cut-link list does not match the solid flags"
        assert np.all((q > 0) & (q <= 1)), "gamma must lie in (0, 1] (Sec. 2)"
        self.link_node, self.link_d, self.link_q, self.link_uw = node, d, q, uw
        self.link_l = l_of_gamma(q, c0, c1, c2)
        # two-node scheme (Eq. 2.11) on the links whose x_l = x_f + e_i is fluid
        self.two_node = bool(two_node)
        self.link_xl = self.nbr[lat.opp[d], node] if len(node) else np.zeros(0, np.int64)
        assert np.all(self.link_l >= 0), "l must be non-negative (Sec. 2)"

        self.f = np.full((lat.Q, self.N), np.nan)
        self.t = 0

    # -- state ------------------------------------------------------------
    def init_equilibrium(self, rho=None, u=None):
        """f = f^eq(rho, u) on fluid nodes (rest state rho0, u = 0 by default)."""
        rho = np.full(self.N, self.rho0) if rho is None else np.asarray(rho, float).reshape(self.N)
        uu = np.zeros((3, self.N))
        if u is not None:
            u = np.asarray(u, float).reshape(self.N, -1)
            uu[: u.shape[1]] = u.T
        f = equilibrium(self.lat, rho, uu, self.rho0)
        f[:, self.solid] = np.nan
        self.f = f
        self.t = 0

    def moments(self):
        """rho and the reported velocity u = j/rho0 + g/2 on fluid nodes (NaN on solid)."""
        rho, j = density_momentum(self.lat, self.f)
        u = j / self.rho0 + 0.5 * self.g[:, None]
        rho = np.where(self.fluid, rho, np.nan)
        u = np.where(self.fluid[None, :], u, np.nan)
        return rho, u.T.copy()

    # -- one step ---------------------------------------------------------
    def step(self, nsteps=1):
        for _ in range(nsteps):
            self._step()

    def _step(self):
        lat = self.lat
        f = self.f
        fl = self.fluid
        # Eq. (2.2a): collision, point-wise, on fluid nodes
        fpost = np.full_like(f, np.nan)
        fpost[:, fl] = collide(lat, f[:, fl], self.S, self.rho0, self.g)
        # Eq. (2.2b): advection f_i(x + e_i, t+1) = f'_i(x, t) between fluid nodes
        fnew = np.full_like(f, np.nan)
        for i in range(lat.Q):
            tgt = self.nbr[i]
            ok = fl & fl[tgt]
            fnew[i, tgt[ok]] = fpost[i, ok]
        # boundary scheme on every cut link (x_f + e_d solid, i = opp(d)); the
        # links are independent, so they are evaluated together, element by element
        n = self.link_node
        d = self.link_d
        i = lat.opp[d]
        nxt = None
        if self.two_node:
            xl = self.link_xl
            nxt = np.where(fl[xl], fpost[d, xl], f[d, n])    # x_l solid: Eq. (2.9)
        fnew[i, n] = boundary_value(
            lat.w[i], lat.e[i], self.link_q, self.link_l, self.b, self.rho0,
            self.link_uw, f[i, n], f[d, n], fpost[i, n], fpost[d, n], nxt)
        assert not np.isnan(fnew[:, fl]).any(), "a fluid population was not written"
        self.f = fnew
        self.t += 1

    def populations(self):
        """f_i(x, t) as (Q, nz, ny, nx); NaN on solid nodes."""
        nx, ny, nz = self.shape
        return self.f.reshape(self.lat.Q, nz, ny, nx).copy()

    def mass(self):
        return float(self.f[:, self.fluid].sum())


def relative_l2_error(u_exact, u_lb, mask):
    """Sec. 3.1, Eq. (eqn:L2-error): sqrt(sum |u - u*|^2) / sqrt(sum |u|^2) over mask."""
    ue = np.asarray(u_exact)[mask]
    ul = np.asarray(u_lb)[mask]
    return float(np.sqrt(((ue - ul) ** 2).sum()) / np.sqrt((ue ** 2).sum()))
