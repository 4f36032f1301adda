"""Full-rank discrete-ordinates (S_N) oracle — TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy restatement of the discretisation the low-rank scheme
approximates:
  * Lie splitting x-advection -> y-advection -> absorption/scattering/source
    (Section 3, the three sub-problems before Section 3.1), or its symmetric
    (Strang) form x(dt/2), y(dt/2), collision(dt), y(dt/2), x(dt/2), the usual
    second-order splitting the same section points to,
  * first-order upwind finite volumes on a uniform cell-centred grid
    (Section 4 introduction; Appendix A), each direction upwinded by the sign of
    its own velocity component, zero inflow at the physical boundary unless
    inflow data f = g(s) h(Omega) are given for a side (the Hohlraum and boundary
    point-source inflow of Section 4),
  * explicit Euler or classic RK4 per sub-step (Section 4 introduction).
Scattering is sigma_s/|S| * rho with rho = sum_q w_q f_q (Eq. (rt) with the
circle's 1/(2 pi) replaced by 1/|S| for a general quadrature).

Pins (tests/test_oracle_sn.py): exact one-cell shift at Courant number 1,
telescoping mass balance, homogeneous isotropic decay factor, source growth.
"""
from __future__ import annotations

import numpy as np


def _integrate(y, rhs, dt, method):
    if method == "euler":
        return y + dt * rhs(y)
    if method == "rk4":
        k1 = rhs(y)
        k2 = rhs(y + 0.5 * dt * k1)
        k3 = rhs(y + 0.5 * dt * k2)
        k4 = rhs(y + dt * k3)
        return y + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    raise ValueError(method)


def advection_rhs(f, omega, axis, h, c_adv=1.0, ghosts=None):
    """-c_adv * omega_q * d/d(axis) f with per-direction upwinding.

    f has shape (ny, nx, n); axis 1 is x, axis 0 is y.  The ghost values outside the
    physical domain are ghosts = (low side, high side), each shaped like one slice of f
    along the axis; None means 0 (zero inflow).  omega_q = 0 gives no flux.
    """
    zero = np.zeros_like(np.take(f, [0], axis=axis))
    g_lo, g_hi = ghosts if ghosts is not None else (zero, zero)
    lo = np.concatenate([g_lo, f], axis=axis)       # lo[c] = f[c-1]
    hi = np.concatenate([f, g_hi], axis=axis)       # hi[c+1] = f[c+1]
    n_ax = f.shape[axis]
    f_prev = np.take(lo, range(0, n_ax), axis=axis)
    f_next = np.take(hi, range(1, n_ax + 1), axis=axis)
    back = (f - f_prev) / h
    fwd = (f_next - f) / h
    pos = omega > 0
    neg = omega < 0
    out = np.zeros_like(f)
    out[..., pos] = -c_adv * omega[pos] * back[..., pos]
    out[..., neg] = -c_adv * omega[neg] * fwd[..., neg]
    return out


def inflow_ghosts(wl, axis):
    """Ghost slices of the physical inflow f(s, Omega) = g(s) h(Omega) along the axis
    (1 = x, 0 = y) for the directions entering through each side: Omega >= 0 at the
    low side, Omega < 0 at the high side (the masks of the subdomain interfaces)."""
    om = wl.omega_x if axis == 1 else wl.omega_y
    out = []
    for side, mask in (("lo", om >= 0), ("hi", om < 0)):
        key = ("x_" if axis == 1 else "y_") + side
        if key in wl.inflow:
            g, hq = wl.inflow[key]
            v = np.asarray(g, dtype=np.float64)[:, None] * (np.asarray(hq, dtype=np.float64) * mask)[None, :]
            out.append(v[:, None, :] if axis == 1 else v[None, :, :])
        else:
            shape = (wl.ny, 1, wl.n) if axis == 1 else (1, wl.nx, wl.n)
            out.append(np.zeros(shape))
    return tuple(out)


def collision_rhs(f, wl):
    """sigma_s/|S| rho - sigma_t f + Q (Eq. (rt) right-hand side)."""
    ssum = float(np.sum(wl.w))
    rho = f @ wl.w                                   # (ny, nx)
    sig_s = wl.sigma_s.reshape(wl.ny, wl.nx)
    sig_t = sig_s + wl.sigma_a.reshape(wl.ny, wl.nx)
    Q = wl.source.reshape(wl.ny, wl.nx)
    return (sig_s * rho / ssum)[..., None] - sig_t[..., None] * f + Q[..., None]


def initial_state(wl):
    return np.repeat(wl.g0.reshape(wl.ny, wl.nx)[..., None], wl.n, axis=2).astype(np.float64)


def step(f, wl, dt=None):
    """One split time step: x-advection, y-advection, collision (Lie), or
    x(dt/2), y(dt/2), collision(dt), y(dt/2), x(dt/2) (Strang)."""
    dt = wl.dt if dt is None else dt
    m = wl.integrator
    gx, gy = inflow_ghosts(wl, 1), inflow_ghosts(wl, 0)
    ax = lambda g, h: _integrate(g, lambda u: advection_rhs(u, wl.omega_x, 1, wl.hx, wl.c_adv, gx), h, m)
    ay = lambda g, h: _integrate(g, lambda u: advection_rhs(u, wl.omega_y, 0, wl.hy, wl.c_adv, gy), h, m)
    co = lambda g, h: _integrate(g, lambda u: collision_rhs(u, wl), h, m)
    if wl.splitting == "strang":
        return ax(ay(co(ay(ax(f, 0.5 * dt), 0.5 * dt), dt), 0.5 * dt), 0.5 * dt)
    return co(ay(ax(f, dt), dt), dt)


def unsplit_rhs(f, wl):
    """The whole semi-discrete right-hand side (no splitting): the reference the
    splittings converge to as dt -> 0."""
    return (advection_rhs(f, wl.omega_x, 1, wl.hx, wl.c_adv, inflow_ghosts(wl, 1))
            + advection_rhs(f, wl.omega_y, 0, wl.hy, wl.c_adv, inflow_ghosts(wl, 0))
            + collision_rhs(f, wl))


def run(wl, nsteps=None, f=None):
    f = initial_state(wl) if f is None else f
    for _ in range(wl.nsteps if nsteps is None else nsteps):
        f = step(f, wl)
    return f


def scalar_flux(f, wl):
    """rho_c = sum_q w_q f_cq, flattened x-fastest (Section 2)."""
    return (f @ wl.w).reshape(-1)
