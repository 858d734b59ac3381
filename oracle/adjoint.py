"""Discrete adjoint of the oracle's time step (TEST INFRASTRUCTURE ONLY).

Reverse-mode differentiation of `lbm.Simulation.step` for the loss
    J = sum over masked fluid nodes of |u(x, T) - u_target(x)|^2,
with u the reported velocity j/rho0 + g/2 after T steps.  Gradients are returned
with respect to the relaxation rates s_k (all Q), every link's wall fraction q
(= gamma of Sec. 2) and wall velocity phi.

It is written independently of the GPU adjoint, in f-space with dense per-node
Jacobians:
* collision (Appendix): f' = f - M^-1 S M (f - f^eq(f)) + const, so
  d f'/d f = I - M^-1 S M (I - d f^eq/d f), with d f^eq_i/d f_k =
  w_i (1 + 3 c_i.c_k + 9 (c_i.u)(c_i.c_k) - 3 u.c_k) from Eq. (42);
* advection (Eq. 2.2b) is a permutation, its transpose a gather;
* boundary (Eq. 2.13) is linear in the four populations it combines; its partial
  derivatives, and those with respect to gamma and phi, are taken from the
  oracle's own `boundary_value` by complex-step differentiation (exact to
  rounding for this rational function), so no coefficient is retyped here.
The forward states are stored in full (small grids only).
"""

import numpy as np

from . import lbm as O
from .lattices import CS2


def _collision_jacobian(lat, f, S, rho0):
    """d f'/d f for every node: (N, Q, Q), Appendix MRT with Eq. (42)."""
    c = lat.e.astype(np.float64)
    rho, j = O.density_momentum(lat, f)
    u = j / rho0                                           # (3, N)
    cu = c @ u                                             # (Q, N)
    cc = c @ c.T                                           # (Q, Q) c_i.c_k
    uc = (c @ u).T                                         # (N, Q) u.c_k
    # d feq_i / d f_k
    Jeq = lat.w[None, :, None] * (1 + 3 * cc[None, :, :] + 9 * cu.T[:, :, None] * cc[None, :, :]
                                  - 3 * uc[:, None, :])
    A = lat.Minv @ np.diag(S) @ lat.M                      # (Q, Q)
    I = np.eye(lat.Q)
    return I[None] - np.einsum("ik,nkl->nil", A, I[None] - Jeq)


def _boundary_partials(sim, k, fi, fd, pi, pd):
    """d f_new/d (f_i, f_d, f'_i, f'_d, gamma, phi) of link k by complex step."""
    lat = sim.lat
    d = sim.link_d[k]
    i = lat.opp[d]
    q = sim.link_q[k]
    h = 1e-30
    args = [fi, fd, pi, pd]
    c0, c1, c2 = sim.scheme_coeffs

    def bv(gamma, phi, vals):
        l = O.l_of_gamma(gamma, c0, c1, c2)
        return O.boundary_value(lat.w[i], lat.e[i], gamma, l, sim.b, sim.rho0, phi, *vals)

    out = []
    for a in range(4):
        vals = [complex(v) for v in args]
        vals[a] += 1j * h
        out.append(bv(complex(q), sim.link_uw[k].astype(complex), vals).imag / h)
    dq = bv(q + 1j * h, sim.link_uw[k].astype(complex), [complex(v) for v in args]).imag / h
    dphi = np.zeros(3)
    for a in range(3):
        phi = sim.link_uw[k].astype(complex)
        phi[a] += 1j * h
        dphi[a] = bv(complex(q), phi, [complex(v) for v in args]).imag / h
    return np.array(out), float(dq), dphi


def adjoint(sim, n_steps, mask, u_target):
    """Run n_steps forward from sim's current state and return
    (J, dJ/ds (Q,), dJ/dq (links,), dJ/dphi (links, 3)).  sim ends advanced."""
    assert not getattr(sim, "two_node", False), "the adjoint follows the single-node scheme"
    lat = sim.lat
    Q, N = lat.Q, sim.N
    fl = sim.fluid
    mask = np.asarray(mask, bool).reshape(N) & fl
    u_target = np.asarray(u_target, float).reshape(N, -1)
    D = u_target.shape[1]
    states = []
    for _ in range(n_steps):
        states.append(sim.f.copy())
        sim.step()
    # loss and its gradient with respect to f(T)
    _, u = sim.moments()
    diff = np.where(mask[:, None], u[:, :D] - u_target, 0.0)
    J = float((diff ** 2).sum())
    c = lat.e.astype(np.float64)
    lam = np.zeros((Q, N))
    lam[:, mask] = (2.0 / sim.rho0) * (c[:, :D] @ diff[mask].T)

    gs = np.zeros(Q)
    gq = np.zeros(len(sim.link_node))
    gphi = np.zeros((len(sim.link_node), 3))
    cut = np.zeros((Q, N), bool)                  # cut[d, n]: link (n, d) exists
    cut[sim.link_d, sim.link_node] = True
    for t in range(n_steps - 1, -1, -1):
        f = states[t]
        fpost = np.full_like(f, np.nan)
        fpost[:, fl] = O.collide(lat, f[:, fl], sim.S, sim.rho0, sim.g)
        lam_post = np.zeros((Q, N))               # adjoint of f'
        lam_pre = np.zeros((Q, N))                # direct adjoint of f (boundary terms)
        # advection transpose: f_{t+1,i}(x + e_i) = f'_i(x) for fluid x, x + e_i
        for i in range(Q):
            tgt = sim.nbr[i]
            ok = fl & fl[tgt]
            lam_post[i, ok] += lam[i, tgt[ok]]
        # boundary transpose
        for k in range(len(sim.link_node)):
            n = sim.link_node[k]
            d = sim.link_d[k]
            i = lat.opp[d]
            part, dq, dphi = _boundary_partials(sim, k, f[i, n], f[d, n], fpost[i, n], fpost[d, n])
            a = lam[i, n]
            lam_pre[i, n] += part[0] * a
            lam_pre[d, n] += part[1] * a
            lam_post[i, n] += part[2] * a
            lam_post[d, n] += part[3] * a
            gq[k] += dq * a
            gphi[k] += dphi * a
        # relaxation-rate gradient: d f'/d s_k = -M^-1 e_k (M (f - feq))_k
        rho, j = O.density_momentum(lat, f[:, fl])
        feq = O.equilibrium(lat, rho, j / sim.rho0, sim.rho0)
        mneq = lat.M @ (f[:, fl] - feq)                       # (Q, Nf)
        mu = lat.Minv.T @ lam_post[:, fl]                      # (Q, Nf)
        gs += -(mu * mneq).sum(axis=1)
        # collision transpose
        Jc = _collision_jacobian(lat, f[:, fl], sim.S, sim.rho0)
        lam_new = lam_pre.copy()
        lam_new[:, fl] += np.einsum("nik,in->kn", Jc, lam_post[:, fl])
        lam = lam_new
    return J, gs, gq, gphi


def loss(sim, n_steps, mask, u_target):
    """Forward only: J after n_steps (sim advanced)."""
    sim.step(n_steps)
    _, u = sim.moments()
    u_target = np.asarray(u_target, float).reshape(sim.N, -1)
    D = u_target.shape[1]
    m = np.asarray(mask, bool).reshape(sim.N) & sim.fluid
    diff = u[m, :D] - u_target[m]
    return float((diff ** 2).sum())
