"""Pins of the full-rank S_N oracle against closed forms (no GPU).

Each test fixes a part of oracle/sn.py by a value the mathematics determines
independently of the code: an exact shift, a telescoping balance, a decay
factor, a source increment.
"""
import math

import numpy as np
import pytest

from oracle import sn
from paper_2602_14854_gb300 import inputs


def axis_workload(nx=6, ny=5, dt=None, integrator="euler"):
    """Four axis-aligned directions (+-1, 0), (0, +-1); weights pi/2."""
    ox = np.array([1.0, -1.0, 0.0, 0.0])
    oy = np.array([0.0, 0.0, 1.0, -1.0])
    w = np.full(4, math.pi / 2)
    nc = nx * ny
    h = 1.0 / nx
    return inputs.Workload(
        name="axis", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=ny * h, xcuts=[0, nx],
        ycuts=[0, ny], omega_x=ox, omega_y=oy, w=w, sigma_s=np.zeros(nc),
        sigma_a=np.zeros(nc), source=np.zeros(nc), g0=np.zeros(nc),
        dt=h if dt is None else dt, nsteps=1, integrator=integrator)


def test_unit_courant_is_exact_shift():
    """Upwind at Courant number 1 moves every direction exactly one cell (zero inflow)."""
    wl = axis_workload()
    rng = np.random.default_rng(0)
    f = rng.uniform(size=(wl.ny, wl.nx, 4))
    fx = sn.step(f, wl)            # x-sweep, y-sweep (sigma = 0, Q = 0: collision is identity)
    expect = np.zeros_like(f)
    # x-sweep: +x shifts right, -x shifts left; then y-sweep: +y shifts up, -y shifts down
    expect[:, 1:, 0] = f[:, :-1, 0]
    expect[:, :-1, 1] = f[:, 1:, 1]
    expect[1:, :, 2] = f[:-1, :, 2]
    expect[:-1, :, 3] = f[1:, :, 3]
    assert np.max(np.abs(fx - expect)) < 1e-15


def test_mass_balance_telescopes():
    """Euler x-sweep: change of mass = -dt * net outflow through the two x faces."""
    wl = inputs.random_small_problem(3, nx=7, ny=5, tiles_x=1, tiles_y=1, n_mu=2, n_phi=8)
    rng = np.random.default_rng(1)
    f = rng.uniform(size=(wl.ny, wl.nx, wl.n))
    dt = 0.3 * wl.hx
    f1 = f + dt * sn.advection_rhs(f, wl.omega_x, 1, wl.hx)
    mass = lambda g: wl.hx * wl.hy * np.sum(g @ wl.w)
    ox = wl.omega_x
    out_right = np.sum(wl.w * np.maximum(ox, 0) * f[:, -1, :].sum(axis=0)) * wl.hy
    out_left = np.sum(wl.w * np.maximum(-ox, 0) * f[:, 0, :].sum(axis=0)) * wl.hy
    assert abs((mass(f1) - mass(f)) + dt * (out_right + out_left)) < 1e-14 * mass(f)


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_isotropic_homogeneous_decay(integrator):
    """Spatially uniform isotropic state: collision multiplies f by the stability
    polynomial of the integrator at -dt*sigma_a (scattering conserves)."""
    wl = inputs.random_small_problem(2, nx=4, ny=4).with_(integrator=integrator)
    nc = wl.ncells
    sa, ss = 0.7, 1.3
    wl = wl.with_(sigma_a=np.full(nc, sa), sigma_s=np.full(nc, ss), source=np.zeros(nc))
    f = np.full((wl.ny, wl.nx, wl.n), 2.5)
    f1 = sn._integrate(f, lambda g: sn.collision_rhs(g, wl), wl.dt, integrator)
    z = -wl.dt * sa
    fac = 1 + z if integrator == "euler" else 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.max(np.abs(f1 - 2.5 * fac)) < 1e-14


def test_decay_converges_to_exponential():
    """Euler decay factor (1 - dt s)^{T/dt} -> exp(-s T) with first-order error."""
    wl0 = inputs.random_small_problem(2, nx=2, ny=2)
    nc = wl0.ncells
    errs = []
    for nst in (20, 40, 80):
        wl = wl0.with_(sigma_a=np.full(nc, 1.0), sigma_s=np.zeros(nc), source=np.zeros(nc),
                       dt=1.0 / nst)
        f = np.ones((2, 2, wl.n))
        for _ in range(nst):
            f = sn._integrate(f, lambda g: sn.collision_rhs(g, wl), wl.dt, "euler")
        errs.append(abs(f[0, 0, 0] - math.exp(-1.0)))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_source_increment():
    """No material, zero data: one step adds exactly dt * |S| * Q to the density."""
    wl = inputs.random_small_problem(5, nx=6, ny=6)
    nc = wl.ncells
    wl = wl.with_(sigma_s=np.zeros(nc), sigma_a=np.zeros(nc))
    f = sn.step(np.zeros((wl.ny, wl.nx, wl.n)), wl)
    rho = sn.scalar_flux(f, wl)
    assert np.max(np.abs(rho - wl.dt * np.sum(wl.w) * wl.source)) < 1e-15


def test_quadrature_weights_and_moments():
    """Product set: weights sum to 4 pi, odd moments vanish, <Omega_x^2> = 4 pi / 3."""
    ox, oy, w = inputs.product_quadrature(8, 16)
    assert abs(np.sum(w) - 4 * math.pi) < 1e-13
    assert abs(np.sum(w * ox)) < 1e-13 and abs(np.sum(w * oy)) < 1e-13
    assert abs(np.sum(w * ox * ox) - 4 * math.pi / 3) < 1e-12
    assert abs(np.sum(w * ox * oy)) < 1e-13


def splitting_errors(splitting, steps=(4, 8, 16), T=0.1):
    """Errors at time T of the split S_N step against the unsplit semi-discrete
    solution (RK4 at a step 1/32 of the finest), for a smooth heterogeneous problem."""
    wl0 = inputs.random_small_problem(3, nx=12, ny=12, n_mu=2, n_phi=8, integrator="rk4")
    f0 = sn.initial_state(wl0)
    nref = 32 * max(steps)
    ref = f0.copy()
    for _ in range(nref):
        ref = sn._integrate(ref, lambda g: sn.unsplit_rhs(g, wl0), T / nref, "rk4")
    errs = []
    for n in steps:
        wl = wl0.with_(dt=T / n, nsteps=n, splitting=splitting)
        f = sn.run(wl, f=f0.copy())
        errs.append(float(np.linalg.norm(f - ref) / np.linalg.norm(ref)))
    return errs


def test_strang_splitting_is_second_order():
    """Section 3: the Lie splitting of x-, y-advection and collision is first order in
    time; its symmetric (Strang) form is second order.  Measured against the unsplit
    semi-discrete solution, halving dt divides the error by ~2 (Lie) and ~4 (Strang)."""
    lie = splitting_errors("lie")
    strang = splitting_errors("strang")
    lie_order = [math.log2(a / b) for a, b in zip(lie, lie[1:])]
    strang_order = [math.log2(a / b) for a, b in zip(strang, strang[1:])]
    assert all(0.8 < p < 1.3 for p in lie_order), lie_order
    assert all(1.8 < p < 2.3 for p in strang_order), strang_order
    assert strang[-1] < 0.2 * lie[-1]


def test_mass_balance_with_inflow():
    """Euler x-sweep with inflow data f = g(y) h(Omega) on both x sides: the change of
    mass equals dt times (inflow through the faces - outflow through the faces), the
    inflow being hy sum_j sum_q w_q |Omega_q| g_j h_q over the entering directions."""
    wl = inputs.random_small_problem(3, nx=7, ny=5, tiles_x=1, tiles_y=1, n_mu=2, n_phi=8)
    rng = np.random.default_rng(2)
    g_lo, g_hi = rng.uniform(size=wl.ny), rng.uniform(size=wl.ny)
    h_lo, h_hi = rng.uniform(size=wl.n), rng.uniform(size=wl.n)
    wl = wl.with_(inflow={"x_lo": (g_lo, h_lo), "x_hi": (g_hi, h_hi)})
    f = rng.uniform(size=(wl.ny, wl.nx, wl.n))
    dt = 0.3 * wl.hx
    f1 = f + dt * sn.advection_rhs(f, wl.omega_x, 1, wl.hx, 1.0, sn.inflow_ghosts(wl, 1))
    mass = lambda u: wl.hx * wl.hy * np.sum(u @ wl.w)
    ox = wl.omega_x
    out_right = np.sum(wl.w * np.maximum(ox, 0) * f[:, -1, :].sum(axis=0)) * wl.hy
    out_left = np.sum(wl.w * np.maximum(-ox, 0) * f[:, 0, :].sum(axis=0)) * wl.hy
    in_left = np.sum(wl.w * np.maximum(ox, 0) * h_lo) * g_lo.sum() * wl.hy
    in_right = np.sum(wl.w * np.maximum(-ox, 0) * h_hi) * g_hi.sum() * wl.hy
    change = mass(f1) - mass(f)
    assert abs(change - dt * (in_left + in_right - out_right - out_left)) < 1e-14 * mass(f)
    assert dt * (in_left + in_right) > 1e-3 * mass(f)      # the inflow term matters
