"""Seeded synthetic inputs: geometries, wall fractions, wall velocities, parameters.

This module generates INPUTS only -- solid flags, the cut-link list (node, direction,
wall fraction q, wall velocity phi), relaxation vectors and analytic reference
fields.  It holds none of the lattice-Boltzmann arithmetic; both the CUDA library
and the FP64 CPU oracle consume what it produces.

Conventions (those of the C-ABI in include/lbm.h):

* grid shape (nx, ny, nz), nz = 1 in 2D; node index n = x + nx*(y + ny*z); node
  (x, y, z) sits at the point (x, y, z) in lattice units;
* all axes are periodic; the x-wrap may be skewed by (sy, sz): the field is
  invariant under the translation (nx, sy, sz);
* a cut link (n, d, q, phi) has the fluid node x_f = x_n, the solid neighbour
  x_f + e_d, the wall point x_b = x_f + q e_d with q in (0, 1] (Sec. 2 of the
  paper writes x_b = x_f - gamma h e_i with e_i = -e_d), and the wall velocity
  phi(x_b);
* a node exactly on a wall is solid, so q = 1 is possible and q = 0 is not.

The direction tables below are the C-ABI's numbering (plain data).
"""


import numpy as np

# C-ABI direction numbering.  D2Q9 and D3Q15 follow the paper's Appendix order;
# D3Q19 is rest, +x,-x,+y,-y,+z,-z, then the twelve edges, each followed by its
# opposite.
DIRECTIONS = {
    "D2Q9": np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
                      (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)], dtype=np.int64),
    "D3Q19": np.array([
        (0, 0, 0),
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.int64),
    # D3Q15 in the paper's Appendix order: rest, faces, then the eight corners
    "D3Q15": np.array([
        (0, 0, 0),
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 1), (-1, 1, 1), (1, -1, 1), (-1, -1, 1),
        (1, 1, -1), (-1, 1, -1), (1, -1, -1), (-1, -1, -1)], dtype=np.int64),
}


def relaxation_rates(lattice, s_nu):
    """Relaxation vector S in the C-ABI's moment order.

    D2Q9: the paper's Sec. 3 prints diag(1, 1.8, 1.2, 1, 0.5, 0.5, 1, s_nu, s_nu),
    which relaxes q_x at 0.5 and q_y at 1 (anisotropic); read as a transposition
    and use (1, 1.8, 1.2, 1, 0.5, 1, 0.5, s_nu, s_nu), the j/q pattern of the
    paper's D3Q15 vector.
    D3Q19 (rows rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, 3pi_xx, p_ww,
    pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z): the paper's D3Q15 choice mapped onto
    these rows; the fourth-order pi moments take 1.2, the third-order m moments 1.5.
    D3Q15 (rows rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, p_ww, p_xy, p_yz,
    p_xz, m_xyz): the vector the paper prints in Sec. 3.
    """
    if lattice == "D2Q9":
        s = [1, 1.8, 1.2, 1, 0.5, 1, 0.5, s_nu, s_nu]
    elif lattice == "D3Q19":
        s = [1, 1.8, 1.2, 1, 0.5, 1, 0.5, 1, 0.5,
             s_nu, 1.2, s_nu, 1.2, s_nu, s_nu, s_nu, 1.5, 1.5, 1.5]
    elif lattice == "D3Q15":
        s = [1, 1.8, 1.2, 1, 0.5, 1, 0.5, 1, 0.5, s_nu, s_nu, s_nu, s_nu, s_nu, 1.5]
    else:
        raise ValueError(lattice)
    return np.array(s, dtype=np.float64)


def relaxation_rates_bgk(lattice, s):
    """BGK (single relaxation time) as an MRT vector: every non-conserved moment
    relaxes at s (the conserved rows' rates have no effect)."""
    Q = len(DIRECTIONS[lattice])
    return np.full(Q, float(s))


def relaxation_rates_trt(lattice, s_plus, magic=3.0 / 16.0):
    """Two-relaxation-time collision as an MRT vector: the rows of M that are even
    under e -> -e relax at s_plus, the odd ones at s_minus, chosen from the "magic"
    product (1/s_plus - 1/2)(1/s_minus - 1/2) = magic.  Every row of the three
    bases is even or odd, so this is exactly the TRT operator."""
    E = DIRECTIONS[lattice]
    Q = len(E)
    # parity of each row: rows whose moment changes sign under e -> -e (odd powers)
    odd = {"D2Q9": [3, 4, 5, 6], "D3Q19": [3, 4, 5, 6, 7, 8, 16, 17, 18],
           "D3Q15": [3, 4, 5, 6, 7, 8, 14]}[lattice]
    s_minus = 1.0 / (magic / (1.0 / s_plus - 0.5) + 0.5)
    s = np.full(Q, float(s_plus))
    s[odd] = s_minus
    return s


def s_nu_for(nu_lattice):
    """Lattice viscosity nu = (1/s_nu - 1/2)/3 (Sec. 3 with eta h^2 = delta_t = 1)."""
    return 1.0 / (3.0 * nu_lattice + 0.5)


def nu_for(s_nu):
    return (1.0 / s_nu - 0.5) / 3.0


# ----------------------------------------------------------------------------
# generic helpers
# ----------------------------------------------------------------------------

def _coords(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def _wrap(shape, skew, X, Y, Z):
    nx, ny, nz = shape
    k = np.floor_divide(X, nx)
    return (X - k * nx) + nx * (np.mod(Y - k * skew[0], ny) + ny * np.mod(Z - k * skew[1], nz))


def _first_root(a, b, c):
    """Smallest root t > 0 of a t^2 + b t + c = 0, clipped to (0, 1]."""
    disc = np.maximum(b * b - 4 * a * c, 0.0)
    sq = np.sqrt(disc)
    t1 = (-b - sq) / (2 * a)
    t2 = (-b + sq) / (2 * a)
    t = np.where(t1 > 0, t1, t2)
    return np.clip(t, 1e-12, 1.0)


def cut_links(lattice, shape, skew, solid):
    """All (n, d) with fluid n and solid n + e_d, sorted by node then direction."""
    E = DIRECTIONS[lattice]
    x, y, z = _coords(shape)
    solid = np.asarray(solid, dtype=bool).ravel()
    fluid = ~solid
    nodes, dirs = [], []
    for d in range(1, len(E)):
        nb = _wrap(shape, skew, x + E[d, 0], y + E[d, 1], z + E[d, 2])
        sel = np.nonzero(fluid & solid[nb])[0]
        nodes.append(sel)
        dirs.append(np.full(len(sel), d, dtype=np.int64))
    node = np.concatenate(nodes)
    d = np.concatenate(dirs)
    order = np.lexsort((d, node))
    return node[order], d[order]


# ----------------------------------------------------------------------------
# 2D: circular Couette flow between two cylinders (configs: 64^2, refinement,
# ensemble) and the paper's straight-wall Poiseuille channel (Sec. 3.1)
# ----------------------------------------------------------------------------

def couette_2d(n, center, R1, R2, U1, lattice="D2Q9"):
    """Annulus R1 < r < R2 on an n x n periodic grid; inner wall turns counter-clockwise
    at speed U1, outer wall at rest.  Fluid iff R1 < r < R2 (a node on a wall is solid).

    Returns dict(shape, skew, solid (N,), links{node,d,q,uw}, u_exact (N,3), nu-free).
    The analytic steady field u_theta(r) = U1 R1 (R2^2/r - r)/(R2^2 - R1^2) is the
    textbook circular Couette solution of the incompressible Navier-Stokes equations.
    """
    shape = (int(n), int(n), 1)
    E = DIRECTIONS[lattice]
    cx, cy = float(center[0]), float(center[1])
    x, y, z = _coords(shape)
    r = np.hypot(x - cx, y - cy)
    solid = ~((r > R1) & (r < R2))
    node, d = cut_links(lattice, shape, (0, 0), solid)
    px = x[node].astype(np.float64)
    py = y[node].astype(np.float64)
    dx = E[d, 0].astype(np.float64)
    dy = E[d, 1].astype(np.float64)
    # which wall: the neighbour's radius (unwrapped; the annulus never reaches the
    # grid edge for the configurations used here)
    rn = np.hypot(px + dx - cx, py + dy - cy)
    inner = rn <= R1
    R = np.where(inner, R1, R2)
    wx, wy = px - cx, py - cy
    a = dx * dx + dy * dy
    b = 2 * (dx * wx + dy * wy)
    c = wx * wx + wy * wy - R * R
    q = _first_root(a, b, c)
    xb = px + q * dx - cx
    yb = py + q * dy - cy
    uw = np.zeros((len(node), 3))
    uw[inner, 0] = -U1 * yb[inner] / R1
    uw[inner, 1] = U1 * xb[inner] / R1
    u_exact = np.full((x.size, 3), np.nan)
    fl = ~solid
    rr = r[fl]
    ut = U1 * R1 * (R2 * R2 / rr - rr) / (R2 * R2 - R1 * R1)
    u_exact[fl, 0] = -ut * (y[fl] - cy) / rr
    u_exact[fl, 1] = ut * (x[fl] - cx) / rr
    u_exact[fl, 2] = 0.0
    return dict(lattice=lattice, shape=shape, skew=(0, 0), solid=solid,
                links=dict(node=node, d=d, q=q, uw=uw), u_exact=u_exact)


def couette_config(n):
    """The 64^2 circular Couette problem scaled to n per side (diffusive scaling).

    64^2: centre (32.3, 31.7), R1 = 10, R2 = 28, U1 = 0.01, nu = 0.05; for other n
    the radii and centre scale with n/64, nu stays 0.05 and U1 scales as 64/n.
    """
    s = n / 64.0
    w = couette_2d(n, (32.3 * s, 31.7 * s), 10.0 * s, 28.0 * s, 0.01 / s)
    w["nu"] = 0.05
    w["s_nu"] = s_nu_for(0.05)
    w["S"] = relaxation_rates("D2Q9", w["s_nu"])
    w["rho0"] = 1.0
    w["force"] = (0.0, 0.0, 0.0)
    return w


def taylor_green_disc(inv_h, s_nu, nu=0.002, U0=0.05, rho0=1.0, lattice="D2Q9", shift=(0.0, 0.0)):
    """The paper's Taylor-Green vortex in the disc (x - 1/2)^2 + (y - 1/2)^2 <= 1/16
    (Sec. 3.2): nu = 0.002, U0 = 0.05, p0 = rho0 c_s^2, h = 1/inv_h, delta_t = eta h^2
    with eta = (1/s_nu - 1/2)/(3 nu), no force.

    Node (i, j) sits at (i h, j h), i, j = 0..inv_h; nodes outside the disc or on its
    rim are solid.  Lattice-unit outputs: the analytic velocity scales by eta h, the
    pressure by (eta h)^2, and rho = rho0 + (p - p0)/c_s^2.  The wall velocity of a
    link is the analytic velocity at its wall point x_b = x_f + q e_d at t = 0; the
    whole field decays as exp(-8 pi^2 nu t), so at step n it is the t = 0 value times
    decay**n (decay = exp(-8 pi^2 nu eta h^2)).  T = 1/U0 is `steps` steps (rounded).

    shift moves the disc by (sx, sy) physical units against the lattice (the velocity
    field is 1-periodic, so the shifted problem has the same analytic solution); with
    a nonzero shift the rim test is the plain distance test (exact ties have measure
    zero), and the disc must stay inside the unit square.
    """
    n = int(inv_h) + 1
    h = 1.0 / inv_h
    shape = (n, n, 1)
    E = DIRECTIONS[lattice]
    x, y, z = _coords(shape)
    X, Y = x * h, y * h
    R = 0.25
    # in units of h the disc is 4((2i - m)^2 + (2j - m)^2) < m^2 with m = inv_h: an
    # exact integer test, so nodes on the rim are solid
    m = int(inv_h)
    cx, cy = 0.5 + float(shift[0]), 0.5 + float(shift[1])
    if shift[0] == 0 and shift[1] == 0:
        solid = ~(4 * ((2 * x - m) ** 2 + (2 * y - m) ** 2) < m * m)
    else:
        assert R + max(abs(shift[0]), abs(shift[1])) < 0.5 - 2 * h
        solid = ~((X - cx) ** 2 + (Y - cy) ** 2 < R * R)
    node, d = cut_links(lattice, shape, (0, 0), solid)
    px, py = X[node], Y[node]
    dx = E[d, 0].astype(np.float64) * h
    dy = E[d, 1].astype(np.float64) * h
    wx, wy = px - cx, py - cy
    q = _first_root(dx * dx + dy * dy, 2 * (dx * wx + dy * wy), wx * wx + wy * wy - R * R)
    xb, yb = px + q * dx, py + q * dy
    eta = (1.0 / s_nu - 0.5) / (3.0 * nu)
    vs = eta * h                                   # physical -> lattice velocity

    def vel(xx, yy):
        return (-U0 * np.cos(2 * np.pi * xx) * np.sin(2 * np.pi * yy),
                U0 * np.cos(2 * np.pi * yy) * np.sin(2 * np.pi * xx))

    uw = np.zeros((len(node), 3))
    ub, vb = vel(xb, yb)
    uw[:, 0], uw[:, 1] = ub * vs, vb * vs
    u0 = np.full((x.size, 3), np.nan)
    fl = ~solid
    ux, uy = vel(X, Y)
    u0[fl, 0], u0[fl, 1], u0[fl, 2] = ux[fl] * vs, uy[fl] * vs, 0.0
    dp = -0.25 * U0 * U0 * (np.cos(4 * np.pi * X) + np.cos(4 * np.pi * Y)) * vs * vs
    rho = np.where(fl, rho0 + 3.0 * dp, rho0)
    dt = eta * h * h
    decay = float(np.exp(-8 * np.pi ** 2 * nu * dt))
    steps = int(round((1.0 / U0) / dt))
    return dict(lattice=lattice, shape=shape, skew=(0, 0), solid=solid,
                links=dict(node=node, d=d, q=q, uw=uw), u_exact=u0, rho_init=rho,
                decay=decay, steps=steps, force=(0.0, 0.0, 0.0),
                S=relaxation_rates(lattice, s_nu), rho0=rho0, s_nu=s_nu)


def poiseuille_2d(Ny, gamma, s_nu, nx=2, nu_phys=0.03, lattice="D2Q9"):
    """The paper's Poiseuille channel (Sec. 3.1): rows j = 0 and j = Ny are solid, rows
    1..Ny-1 are fluid, the walls sit a fraction gamma of a link outside rows 1 and
    Ny-1, h = H/(Ny - 2 + 2 gamma), H = 1, nu = 0.03, G = 0.8 nu, delta_t = eta h^2
    with eta = (1/s_nu - 1/2)/(3 nu).  x is periodic (the flow does not depend on x).

    Returns lattice-unit inputs: force g_lat = G eta^2 h^3 along x and the exact
    lattice velocity u_lat = u_phys eta h.
    """
    shape = (int(nx), int(Ny) + 1, 1)
    x, y, z = _coords(shape)
    solid = (y == 0) | (y == Ny)
    node, d = cut_links(lattice, shape, (0, 0), solid)
    q = np.full(len(node), float(gamma))      # every cut link crosses a wall at gamma
    uw = np.zeros((len(node), 3))
    H = 1.0
    h = H / (Ny - 2 + 2 * gamma)
    eta = (1.0 / s_nu - 0.5) / (3.0 * nu_phys)
    G = 0.8 * nu_phys
    g_lat = G * eta * eta * h ** 3
    yy = (y - 1 + gamma) * h                   # distance from the lower wall, physical
    U = G * H * H / (8 * nu_phys)
    u_phys = 4 * U * (1 - yy / H) * (yy / H)
    u_exact = np.full((x.size, 3), np.nan)
    fl = ~solid
    u_exact[fl, 0] = u_phys[fl] * eta * h
    u_exact[fl, 1:] = 0.0
    return dict(lattice=lattice, shape=shape, skew=(0, 0), solid=solid,
                links=dict(node=node, d=d, q=q, uw=uw), u_exact=u_exact,
                force=(g_lat, 0.0, 0.0), S=relaxation_rates(lattice, s_nu), rho0=1.0,
                s_nu=s_nu)


# ----------------------------------------------------------------------------
# 3D: body-force driven flow in a tilted periodic pipe; sphere in a periodic box
# ----------------------------------------------------------------------------

def tilted_pipe_3d(L, radius_frac=0.4, axis_dir=(16, 4, 3), offset=(0.37, 0.21),
                   s_nu=1.0, u_max=None, lattice="D3Q19"):
    """Circular pipe of radius radius_frac*L in an L^3 box, axis parallel to axis_dir.

    axis_dir = (16, 4, 3) tilts the axis by atan(5/16) = 17.4 deg from x overall
    (14.0 deg toward y, 10.6 deg toward z).  The x-wrap is skewed by
    (sy, sz) = (L*4/16, L*3/16) so that the pipe is periodic along its axis;
    y and z wrap plainly, which repeats the pipe at (0, +-L, 0), (0, 0, +-L).
    The axis passes through (L/2, L/2 + offset[0], L/2 + offset[1]).

    Body force g along the axis; the analytic field is the Hagen-Poiseuille profile
    u = U (1 - r^2/R^2) with U = g R^2/(4 nu) (Sec. 3.3, rotated).  By default g
    is chosen so that U = 0.347/L, the lattice velocity of the paper's pipe
    (nu = 0.03, G = 0.8 nu, R = 1/2) at s_nu = 1 and R = 0.4 L.
    """
    L = int(L)
    ad = np.asarray(axis_dir, dtype=np.float64)
    assert (L * axis_dir[1]) % axis_dir[0] == 0 and (L * axis_dir[2]) % axis_dir[0] == 0
    skew = (L * axis_dir[1] // axis_dir[0], L * axis_dir[2] // axis_dir[0])
    a = ad / np.linalg.norm(ad)
    R = radius_frac * L
    shape = (L, L, L)
    c0 = np.array([L / 2, L / 2 + offset[0], L / 2 + offset[1]])
    x, y, z = _coords(shape)
    P = np.stack([x, y, z], axis=1).astype(np.float64)
    images = [np.array([0.0, my * L, mz * L]) for my in (-1, 0, 1) for mz in (-1, 0, 1)]

    def perp(v):
        return v - (v @ a)[:, None] * a[None, :]

    # nearest axis image of every node
    best = np.full(len(P), np.inf)
    best_img = np.zeros(len(P), dtype=np.int64)
    for k, im in enumerate(images):
        dv = perp(P - (c0 + im))
        d2 = (dv * dv).sum(1)
        upd = d2 < best
        best[upd] = d2[upd]
        best_img[upd] = k
    r = np.sqrt(best)
    solid = ~(r < R)
    node, d = cut_links(lattice, shape, skew, solid)
    E = DIRECTIONS[lattice].astype(np.float64)
    centres = np.stack([c0 + im for im in images])[best_img[node]]
    w = perp(P[node] - centres)
    dv = perp(E[d])
    qa = (dv * dv).sum(1)
    qb = 2 * (dv * w).sum(1)
    qc = (w * w).sum(1) - R * R
    q = _first_root(qa, qb, qc)
    uw = np.zeros((len(node), 3))
    nu = nu_for(s_nu)
    if u_max is None:
        u_max = 0.347 / L
    g = 4 * nu * u_max / (R * R)
    u_exact = np.full((x.size, 3), np.nan)
    fl = ~solid
    prof = u_max * (1 - r[fl] ** 2 / (R * R))
    u_exact[fl] = prof[:, None] * a[None, :]
    return dict(lattice=lattice, shape=shape, skew=skew, solid=solid,
                links=dict(node=node, d=d, q=q, uw=uw), u_exact=u_exact,
                force=tuple(g * a), S=relaxation_rates(lattice, s_nu), rho0=1.0,
                s_nu=s_nu, radius=R, axis=a)


def sphere_3d(n, radius, center, s_nu=1.0, force=(1e-6, 0.0, 0.0), lattice="D3Q19"):
    """A solid sphere in a periodic n^3 box (fluid outside, wall at rest)."""
    shape = (int(n),) * 3
    x, y, z = _coords(shape)
    c = np.asarray(center, dtype=np.float64)
    P = np.stack([x, y, z], axis=1).astype(np.float64)
    r = np.linalg.norm(P - c, axis=1)
    solid = r <= radius
    node, d = cut_links(lattice, shape, (0, 0), solid)
    E = DIRECTIONS[lattice].astype(np.float64)
    w = P[node] - c
    dv = E[d]
    q = _first_root((dv * dv).sum(1), 2 * (dv * w).sum(1), (w * w).sum(1) - radius * radius)
    uw = np.zeros((len(node), 3))
    return dict(lattice=lattice, shape=shape, skew=(0, 0), solid=solid,
                links=dict(node=node, d=d, q=q, uw=uw), force=tuple(force),
                S=relaxation_rates(lattice, s_nu), rho0=1.0, s_nu=s_nu)


# ----------------------------------------------------------------------------
# random perturbations used by parity tests (populations away from equilibrium)
# ----------------------------------------------------------------------------

def random_links_uw(links, scale, seed):
    """Replace the wall velocities by seeded random vectors (tests of the wall term)."""
    rng = np.random.default_rng(seed)
    out = dict(links)
    out["uw"] = scale * rng.standard_normal((len(links["node"]), 3))
    return out


def random_state(shape, lattice, rho0, du, seed):
    """Seeded density and velocity fields rho0 + O(du), O(du) for equilibrium starts."""
    rng = np.random.default_rng(seed)
    N = shape[0] * shape[1] * shape[2]
    D = 2 if lattice == "D2Q9" else 3
    rho = rho0 + du * rng.standard_normal(N)
    u = np.zeros((N, 3))
    u[:, :D] = du * rng.standard_normal((N, D))
    return rho, u


def couette_ensemble(count=96, seed=0):
    """Seeded ensemble of circular Couette instances of uneven size.

    Draw order per instance: n ~ U{48..768}, R1/n ~ U(0.1, 0.25), R2/n ~ U(0.35, 0.45),
    U1 ~ U(0.005, 0.02), nu ~ U(0.02, 0.2), centre offset ~ U[0, 1)^2; centre = n/2 + offset.
    Returns a list of parameter dicts (geometry is built on demand by couette_2d).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(48, 769))
        r1 = float(rng.uniform(0.1, 0.25))
        r2 = float(rng.uniform(0.35, 0.45))
        U1 = float(rng.uniform(0.005, 0.02))
        nu = float(rng.uniform(0.02, 0.2))
        o = rng.uniform(0.0, 1.0, size=2)
        out.append(dict(n=n, R1=r1 * n, R2=r2 * n, U1=U1, nu=nu,
                        center=(n / 2 + float(o[0]), n / 2 + float(o[1]))))
    return out


def ensemble_member(p, lattice="D2Q9"):
    """Inputs of one ensemble instance (a dict of couette_ensemble)."""
    w = couette_2d(p["n"], p["center"], p["R1"], p["R2"], p["U1"], lattice)
    w["nu"] = p["nu"]
    w["s_nu"] = s_nu_for(p["nu"])
    w["S"] = relaxation_rates(lattice, w["s_nu"])
    w["rho0"] = 1.0
    w["force"] = (0.0, 0.0, 0.0)
    return w


def fluid_count(solid):
    return int((~np.asarray(solid, dtype=bool)).sum())


def pipe_mlups_units(L):
    """Fluid nodes of the L^3 tilted pipe (the unit the throughput metric counts)."""
    return fluid_count(tilted_pipe_3d(L)["solid"])


