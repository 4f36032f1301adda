"""Pins of the DD-DLRA oracle (no GPU).

Every test fixes part of oracle/dd_dlra.py against something other than the
oracle itself: the full-rank S_N operator written out here, exact identities
of the projector-splitting integrator at full rank, closed-form decay factors,
exact source increments, invariances, reflection symmetry, and convergence to
S_N as the rank grows.
"""
import math

import numpy as np
import pytest

from oracle import dd_dlra, sn
from paper_2602_14854_gb300 import inputs


def circle_problem(nx=8, ny=8, tiles=2, n_phi=8, rank=8, integrator="euler", seed=0):
    """Small heterogeneous problem on the paper's circle quadrature."""
    wl = inputs.random_small_problem(seed, nx=nx, ny=ny, tiles_x=tiles, tiles_y=tiles,
                                     n_mu=0, n_phi=n_phi, rank=rank,
                                     r_aug_max=rank, integrator=integrator)
    return wl


def random_state(o, rank, seed):
    facs = []
    for s in o.subs:
        U, S, V = inputs.random_factors(seed + s.k, s.N, o.wl.n, rank, o.hx, o.hy, o.w)
        facs.append((U, S, V))
    o.set_state(facs)


def upwind_local(f, ox, nyk, nxk, h, g_lo, g_hi, axis):
    """Per-direction upwind advection of f (N_k, n) with ghost rows g_lo/g_hi
    (lines, n), written out independently of the oracle."""
    n = f.shape[1]
    F = f.reshape(nyk, nxk, n)
    if axis == "y":
        F = F.transpose(1, 0, 2)
    out = np.zeros_like(F)
    for q in range(n):
        if ox[q] > 0:
            prev = np.concatenate([g_lo[:, None, q], F[:, :-1, q]], axis=1)
            out[:, :, q] = -ox[q] * (F[:, :, q] - prev) / h
        elif ox[q] < 0:
            nxt = np.concatenate([F[:, 1:, q], g_hi[:, None, q]], axis=1)
            out[:, :, q] = -ox[q] * (nxt - F[:, :, q]) / h
    if axis == "y":
        out = out.transpose(1, 0, 2)
    return out.reshape(-1, n)


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("tiles,integrator", [(2, "euler"), (1, "rk4")])
def test_full_rank_kstep_equals_sn(axis, tiles, integrator):
    """At full rank the K-step of Algorithms 1/2 with the upwind rule of
    Appendix A and the boundary data of Eq. (generate_Kboundary) reproduces the
    S_N sub-step exactly (Euler across interfaces; RK4 on one subdomain, where
    the frozen boundary data is the zero inflow)."""
    wl = circle_problem(tiles=tiles, integrator=integrator)
    o = dd_dlra.DDDLRA(wl, tau=1e-12)
    random_state(o, wl.n, 10)
    f0 = o.full_f()
    snap = o.state
    f1 = np.zeros((wl.ncells, wl.n))
    for k, sub in enumerate(o.subs):
        K0, Vh, info = o.augment(k, axis, snap)
        assert info["r_t"] == wl.n
        lo, hi = o.boundary(k, axis, snap, K0, Vh)
        om = wl.omega_x if axis == "x" else wl.omega_y
        C = Vh.T @ (wl.w[:, None] * om[:, None] * Vh)
        K1 = dd_dlra.integrate(K0, lambda K: o.kstep_rhs_adv(K, C, lo, hi, sub, axis),
                               wl.dt, integrator)
        f1[o.cells[k]] = K1 @ Vh.T
    om, ax, h = (wl.omega_x, 1, wl.hx) if axis == "x" else (wl.omega_y, 0, wl.hy)
    ref = sn._integrate(f0, lambda g: sn.advection_rhs(g, om, ax, h), wl.dt, integrator)
    assert np.max(np.abs(f1.reshape(ref.shape) - ref)) < 1e-12 * np.max(np.abs(ref))


def with_random_inflow(wl, seed=11):
    rng = np.random.default_rng(seed)
    return wl.with_(inflow={"x_lo": (rng.uniform(size=wl.ny), rng.uniform(size=wl.n)),
                            "x_hi": (rng.uniform(size=wl.ny), rng.uniform(size=wl.n)),
                            "y_lo": (rng.uniform(size=wl.nx), rng.uniform(size=wl.n)),
                            "y_hi": (rng.uniform(size=wl.nx), rng.uniform(size=wl.n))})


@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("tiles,integrator", [(2, "euler"), (1, "rk4")])
def test_full_rank_kstep_with_inflow_equals_sn(axis, tiles, integrator):
    """R22: with inflow data f = g(s) h(Omega) on all four physical sides, the
    full-rank K-step (ghost = the inflow's projection for boundary faces, neighbour
    data inside) reproduces the S_N sub-step with the same inflow ghosts."""
    wl = with_random_inflow(circle_problem(tiles=tiles, integrator=integrator))
    o = dd_dlra.DDDLRA(wl, tau=1e-12)
    random_state(o, wl.n, 10)
    f0 = o.full_f()
    snap = o.state
    f1 = np.zeros((wl.ncells, wl.n))
    for k, sub in enumerate(o.subs):
        K0, Vh, info = o.augment(k, axis, snap)
        assert info["r_t"] == wl.n
        lo, hi = o.boundary(k, axis, snap, K0, Vh)
        om = wl.omega_x if axis == "x" else wl.omega_y
        C = Vh.T @ (wl.w[:, None] * om[:, None] * Vh)
        K1 = dd_dlra.integrate(K0, lambda K: o.kstep_rhs_adv(K, C, lo, hi, sub, axis),
                               wl.dt, integrator)
        f1[o.cells[k]] = K1 @ Vh.T
    om, ax, h = (wl.omega_x, 1, wl.hx) if axis == "x" else (wl.omega_y, 0, wl.hy)
    ref = sn._integrate(f0, lambda g: sn.advection_rhs(g, om, ax, h, 1.0,
                                                        sn.inflow_ghosts(wl, ax)),
                        wl.dt, integrator)
    assert np.max(np.abs(f1.reshape(ref.shape) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_inflow_enters_through_the_augmentation():
    """R22: an inflow whose angular profile (peaked around Omega_x = 1) the completion
    families represent poorly is carried into V_hat by its augmentation column: from a
    zero state at rank 4, after three RK4 steps the scalar flux is 6x closer to S_N with
    the column than without it, and the stored ranks stay at the floor."""
    base = inputs.random_small_problem(8, nx=12, ny=12, tiles_x=2, tiles_y=2, n_mu=2,
                                       n_phi=8, rank=4, r_aug_max=8, integrator="rk4",
                                       nsteps=3)
    nc = base.ncells
    om = base.omega_x
    h = np.where(om >= 0, np.exp(-20.0 * (1.0 - om) ** 2), 0.0)
    wl = base.with_(sigma_s=np.zeros(nc), sigma_a=np.zeros(nc), source=np.zeros(nc),
                    g0=np.zeros(nc), inflow={"x_lo": (np.ones(base.ny), h)})
    ref = sn.scalar_flux(sn.run(wl), wl)
    err = lambda o: np.linalg.norm(o.scalar_flux() - ref) / np.linalg.norm(ref)
    with_col = dd_dlra.DDDLRA(wl).run()
    without = dd_dlra.DDDLRA(wl)
    without._inflow_column = lambda *args: None
    without.run()
    assert err(with_col) < 5e-3
    assert err(with_col) < 0.3 * err(without)
    assert all(r == 4 for r in with_col.ranks())


@pytest.mark.parametrize("axis", ["x", "y"])
def test_full_rank_psi_identity(axis):
    """At full rank, explicit Euler K-, S- and L-steps give
    f3 = f1 - dt^2 P_U A_lin(P_U A(f1)), with A the per-direction upwind operator
    (ghost values K^b V^T, frozen) and P_U the weighted projector on the new
    spatial basis: the S-step undoes the projected update and the L-step redoes
    it on the updated data (Eqs. (Sstep_general), (Lstep_general))."""
    wl = circle_problem(tiles=2, integrator="euler")
    o = dd_dlra.DDDLRA(wl, tau=1e-12)
    random_state(o, wl.n, 20)
    snap = o.state
    om = wl.omega_x if axis == "x" else wl.omega_y
    h = wl.hx if axis == "x" else wl.hy
    for k, sub in enumerate(o.subs):
        K0, Vh, _ = o.augment(k, axis, snap)
        lo, hi = o.boundary(k, axis, snap, K0, Vh)
        C = Vh.T @ (wl.w[:, None] * om[:, None] * Vh)
        K1 = K0 + wl.dt * o.kstep_rhs_adv(K0, C, lo, hi, sub, axis)
        U1, S3, V1, _ = o.psi_advection(k, axis, K0, Vh, lo, hi)
        f1 = K1 @ Vh.T
        f3 = U1 @ S3 @ V1.T
        g_lo, g_hi = lo @ Vh.T, hi @ Vh.T
        A = lambda f: upwind_local(f, om, sub.nyk, sub.nxk, h, g_lo, g_hi, axis)
        Z = np.zeros_like(g_lo)
        A_lin = lambda f: upwind_local(f, om, sub.nyk, sub.nxk, h, Z, Z, axis)
        P = lambda f: U1 @ (wl.hx * wl.hy * (U1.T @ f))
        expect = f1 - wl.dt ** 2 * P(A_lin(P(A(f1))))
        assert np.max(np.abs(f3 - expect)) < 1e-11 * np.max(np.abs(f1))


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_kstep_one_signed_directions(sign):
    """Appendix A with a direction set whose x-velocities all have one sign: C is
    definite, so the upwind rule is a plain backward (forward) difference of K
    times C, ghost on the inflow side."""
    rng = np.random.default_rng(3)
    n = 6
    ox = sign * rng.uniform(0.2, 1.0, n)
    oy = rng.uniform(-1, 1, n)
    w = rng.uniform(0.5, 1.5, n)
    nx, ny = 5, 4
    nc = nx * ny
    wl = inputs.Workload(name="half", nx=nx, ny=ny, x0=0, x1=1, y0=0, y1=0.8, xcuts=[0, nx],
                         ycuts=[0, ny], omega_x=ox, omega_y=oy, w=w,
                         sigma_s=np.zeros(nc), sigma_a=np.zeros(nc), source=np.zeros(nc),
                         g0=np.ones(nc), dt=0.1, nsteps=1, rank=3, r_aug_max=3)
    o = dd_dlra.DDDLRA(wl)
    sub = o.subs[0]
    V = np.linalg.qr(rng.standard_normal((n, 3)))[0] / np.sqrt(w)[:, None]
    C = V.T @ (w[:, None] * ox[:, None] * V)
    K = rng.standard_normal((nc, 3))
    glo, ghi = rng.standard_normal((ny, 3)), rng.standard_normal((ny, 3))
    R = o.kstep_rhs_adv(K, C, glo, ghi, sub, "x")
    K3 = K.reshape(ny, nx, 3)
    if sign > 0:
        prev = np.concatenate([glo[:, None, :], K3[:, :-1, :]], axis=1)
        D = (K3 - prev) / wl.hx
    else:
        nxt = np.concatenate([K3[:, 1:, :], ghi[:, None, :]], axis=1)
        D = (nxt - K3) / wl.hx
    assert np.max(np.abs(R - (-(D.reshape(nc, 3) @ C)))) < 1e-12 * np.max(np.abs(R))


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_collision_isotropic_factor(integrator):
    """Homogeneous medium, isotropic rank-1 state: Algorithm 3 multiplies the
    density by R(-x)^2 R(x), x = dt sigma_a, R the integrator's stability
    polynomial (K-step and L-step decay, the minus-signed S-step grows)."""
    wl = inputs.random_small_problem(4, nx=6, ny=6, tiles_x=1, tiles_y=1, rank=1,
                                     r_aug_max=1, integrator=integrator)
    nc = wl.ncells
    sa, ss = 0.8, 1.7
    wl = wl.with_(sigma_a=np.full(nc, sa), sigma_s=np.full(nc, ss), source=np.zeros(nc))
    o = dd_dlra.DDDLRA(wl)
    rho0 = o.scalar_flux()
    o.collision_phase()
    x = wl.dt * sa
    R = (lambda z: 1 + z) if integrator == "euler" else \
        (lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)
    fac = R(-x) ** 2 * R(x)
    assert np.max(np.abs(o.scalar_flux() - fac * rho0)) < 1e-13 * np.max(rho0)


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_source_enters_zero_state(integrator):
    """No material, zero initial data: one full step gives rho = dt |S| Q exactly
    (the collision step starts from the rank floor, completed isotropic-first)."""
    wl = inputs.random_small_problem(6, nx=8, ny=8, integrator=integrator)
    nc = wl.ncells
    wl = wl.with_(sigma_s=np.zeros(nc), sigma_a=np.zeros(nc), g0=np.zeros(nc))
    o = dd_dlra.DDDLRA(wl)
    assert o.ranks() == [0, 0, 0, 0]
    o.step()
    expect = wl.dt * np.sum(wl.w) * wl.source
    assert np.max(np.abs(o.scalar_flux() - expect)) < 1e-14


def test_reparametrisation_invariance():
    """The step depends only on f = U S V^T: (U Th, Th^T S Ph, V Ph) with orthogonal
    Th, Ph gives the same f (augmentation, QR, truncation and completion are
    span-based)."""
    wl = inputs.random_small_problem(7, nx=8, ny=8, n_mu=2, n_phi=8, rank=3, r_aug_max=6,
                                     integrator="rk4")
    a = dd_dlra.DDDLRA(wl)
    b = dd_dlra.DDDLRA(wl)
    random_state(a, 3, 30)
    rng = np.random.default_rng(8)
    rot = []
    for (U, S, V) in a.state:
        Th = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        Ph = np.linalg.qr(rng.standard_normal((3, 3)))[0]
        rot.append((U @ Th, Th.T @ S @ Ph, V @ Ph))
    b.set_state(rot)
    for _ in range(2):
        a.step()
        b.step()
    fa, fb = a.full_f(), b.full_f()
    assert a.ranks() == b.ranks()
    assert np.max(np.abs(fa - fb)) < 1e-11 * np.max(np.abs(fa))


def test_reflection_symmetry():
    """Symmetric data, tiling and quadrature: the density is mirror-symmetric in x
    and in y (Lie splitting keeps each axis' reflection)."""
    wl = inputs.config_c0(integrator="rk4", nsteps=4)
    o = dd_dlra.DDDLRA(wl).run()
    rho = o.scalar_flux().reshape(wl.ny, wl.nx)
    scale = np.max(np.abs(rho))
    assert np.max(np.abs(rho - rho[:, ::-1])) < 1e-11 * scale
    assert np.max(np.abs(rho - rho[::-1, :])) < 1e-11 * scale


def test_rank_convergence_to_sn():
    """One subdomain, RK4: the error against S_N falls as the rank grows
    (Section 2: the low-rank ansatz converges to the full solution)."""
    base = inputs.config_c0(integrator="rk4", tiles_x=1, tiles_y=1, nsteps=12)
    ref = sn.scalar_flux(sn.run(base), base)
    errs = []
    for r in (5, 10, 20, 40):
        wl = base.with_(rank=r, r_aug_max=min(2 * r, base.n))
        rho = dd_dlra.DDDLRA(wl).run().scalar_flux()
        errs.append(np.linalg.norm(rho - ref) / np.linalg.norm(ref))
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[-1] < 1e-3, errs


def test_truncation_tail_rule():
    """Algorithm 5: r' is the smallest rank whose discarded tail is <= tol, and the
    discarded part of f has exactly that norm."""
    wl = inputs.random_small_problem(9, nx=4, ny=4, tiles_x=1, tiles_y=1).with_(
        rank_mode="tol", tol=0.0015, r_min=1, r_max=10)
    o = dd_dlra.DDDLRA(wl)
    rng = np.random.default_rng(2)
    U, _, V = inputs.random_factors(1, 16, wl.n, 5, wl.hx, wl.hy, wl.w)
    P = np.linalg.qr(rng.standard_normal((5, 5)))[0]
    Qm = np.linalg.qr(rng.standard_normal((5, 5)))[0]
    sig = np.array([1.0, 0.1, 0.01, 1e-3, 1e-4])
    S = P @ np.diag(sig) @ Qm.T
    U1, S1, V1 = o.truncate(U, S, V)
    assert S1.shape == (3, 3)
    f = U @ S @ V.T
    f1 = U1 @ S1 @ V1.T
    err = math.sqrt(wl.hx * wl.hy * np.sum((f - f1) ** 2 * wl.w[None, :]))
    assert abs(err - math.hypot(1e-3, 1e-4)) < 1e-14


def test_augmentation_preserves_f():
    """Algorithm 4 keeps F^0 = U S V^T whenever the augmented basis contains V."""
    wl = inputs.random_small_problem(11, nx=8, ny=8, n_mu=2, n_phi=8, rank=3, r_aug_max=9)
    o = dd_dlra.DDDLRA(wl)
    random_state(o, 3, 40)
    for k in range(4):
        for axis in ("x", "y"):
            K0, Vh, info = o.augment(k, axis, o.state)
            assert info["r_t"] == 6          # own 3 + one neighbour's 3 (2x2 tiling)
            U, S, V = o.state[k]
            assert np.max(np.abs(K0 @ Vh.T - U @ S @ V.T)) < 1e-12


def test_outputs_are_weighted_orthonormal():
    wl = inputs.random_small_problem(12, nx=8, ny=8, n_mu=2, n_phi=8, rank=3, r_aug_max=6)
    o = dd_dlra.DDDLRA(wl)
    o.run(2)
    for (U, S, V) in o.state:
        r = S.shape[0]
        assert np.max(np.abs(wl.hx * wl.hy * U.T @ U - np.eye(r))) < 1e-12
        assert np.max(np.abs(V.T @ (wl.w[:, None] * V) - np.eye(r))) < 1e-12


def test_completion_families_orthogonal():
    """The completion families are exactly orthogonal: DCT-II products on the cell
    grid, and P_2l(mu) cos/sin(m phi) under the Gauss-Legendre x equidistant weights."""
    sub = dd_dlra.Sub(0, 0, 0, 0, 6, 0, 5)
    A = np.array(list(dd_dlra.spatial_candidates(sub)))
    G = A @ A.T
    assert A.shape[0] == 30
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-12
    wl = inputs.config_c0()
    cands = []
    for c in dd_dlra.angular_candidates(wl):
        if np.count_nonzero(c) == 1:
            break
        cands.append(c)
    B = np.array(cands)
    assert B.shape[0] == wl.n // 2
    G = B @ (wl.w[:, None] * B.T)
    assert np.max(np.abs(G - np.diag(np.diag(G)))) < 1e-12
    assert np.all(np.diag(G) > 1e-3)
    # isotropic first, then the first azimuthal pair
    assert np.allclose(B[0], 1.0)


def transport_only(tiles, fix, rmin=4):
    return inputs.compact_transport_problem(tiles=tiles, r_min=rmin, mass_fix=fix)


def mass_drift(wl):
    o = dd_dlra.DDDLRA(wl)
    m0 = o.scalar_flux().sum()
    o.run()
    return abs(o.scalar_flux().sum() - m0) / m0


def test_mass_fix_conserves_mass_on_one_subdomain():
    """R18: on one subdomain the K-steps conserve the total mass exactly (no interface,
    nothing reaches the boundary); with the correction the step's mass is theirs.  At
    rank 1 nothing is truncated away and the total mass is conserved to roundoff;
    without the correction the S- and L-steps change it at O(dt^2)."""
    assert mass_drift(transport_only(1, True, rmin=1)) < 1e-12
    assert mass_drift(transport_only(1, False, rmin=1)) > 1e-2


def test_mass_fix_reduces_mass_drift_at_rank_four():
    """Rank floor 4: the truncation of the corrected state drops directions below the
    rank threshold, so conservation is up to that loss, far below the drift without."""
    fixed = mass_drift(transport_only(1, True, rmin=4))
    plain = mass_drift(transport_only(1, False, rmin=4))
    assert fixed < 1e-3 * plain


def test_mass_correction_adds_exactly_delta():
    """R18's correction term: adding delta (x) 1/|S| raises every cell's scalar flux by
    delta (sum_q w_q / |S| = 1) and leaves the rest of f alone; with room under the rank
    cap the truncation keeps it whole.  A zero delta leaves the factors untouched."""
    o = dd_dlra.DDDLRA(transport_only(2, False)).run(1)
    rng = np.random.default_rng(5)
    before = [o._mass(U, S, V, k) for k, (U, S, V) in enumerate(o.state)]
    f_before = [U @ S @ V.T for U, S, V in o.state]
    deltas = [0.1 * np.max(np.abs(m)) * rng.standard_normal(m.shape) for m in before]
    deltas[1] = np.zeros_like(deltas[1])
    kept = o.state[1]
    o.mass_correction(deltas)
    assert all(a is b for a, b in zip(o.state[1], kept))
    for k, (U, S, V) in enumerate(o.state):
        after = o._mass(U, S, V, k)
        scale = np.max(np.abs(before[k])) + np.max(np.abs(deltas[k]))
        assert np.max(np.abs(after - before[k] - deltas[k])) < 1e-12 * scale
        df = U @ S @ V.T - f_before[k]
        iso = np.outer(deltas[k], np.full(V.shape[0], 1.0 / o.ssum))
        assert np.max(np.abs(df - iso)) < 1e-12 * scale


def test_strang_splitting_is_second_order_on_one_subdomain():
    """R20: on one subdomain at full angular rank with RK4 sub-steps the projector
    splitting adds no first-order error, so DD-DLRA inherits the order of the phase
    splitting: against the unsplit semi-discrete S_N solution, halving dt divides the
    scalar-flux error by ~2 with the Lie order of Algorithm 6 and by ~4 with Strang."""
    T = 0.1
    wl0 = inputs.random_small_problem(3, nx=12, ny=12, tiles_x=1, tiles_y=1, n_mu=2,
                                      n_phi=8, integrator="rk4", rank=16, r_aug_max=16)
    f = sn.initial_state(wl0)
    nref = 512
    for _ in range(nref):
        f = sn._integrate(f, lambda g: sn.unsplit_rhs(g, wl0), T / nref, "rk4")
    ref = sn.scalar_flux(f, wl0)
    orders = {}
    for sp in ("lie", "strang"):
        e = []
        for n in (4, 8, 16):
            o = dd_dlra.DDDLRA(wl0.with_(dt=T / n, nsteps=n, splitting=sp)).run()
            e.append(np.linalg.norm(o.scalar_flux() - ref) / np.linalg.norm(ref))
        orders[sp] = [math.log2(a / b) for a, b in zip(e, e[1:])]
    assert all(0.8 < p < 1.3 for p in orders["lie"]), orders
    assert all(1.8 < p < 2.3 for p in orders["strang"]), orders


def test_flux_split_equals_eigen_split_at_full_rank():
    """R21: at full angular rank the eigenvectors of C = <V, Omega V> are the directions
    themselves, so the direction split and Appendix A's eigen-split give the same C+-
    and the same steps (2x2 tiling, RK4)."""
    wl = inputs.random_small_problem(6, nx=8, ny=8, n_mu=2, n_phi=8, rank=16, r_aug_max=16,
                                     integrator="rk4", nsteps=2)
    a = dd_dlra.DDDLRA(wl).run()
    b = dd_dlra.DDDLRA(wl.with_(kstep_split="flux")).run()
    assert a.ranks() == b.ranks()
    ra, rb = a.scalar_flux(), b.scalar_flux()
    assert np.linalg.norm(ra - rb) / np.linalg.norm(ra) < 1e-11


def test_flux_split_kstep_is_energy_stable():
    """R21: with C+ = <V, Omega+ V> positive and C- = <V, Omega- V> negative
    semidefinite and zero inflow, the semi-discrete flux-split K-step cannot create
    energy: <K, R(K)>_x <= 0 for any K.  Swapping the two differences (a plausible
    mistake) creates energy for some K."""
    wl = inputs.random_small_problem(7, nx=8, ny=8, tiles_x=1, tiles_y=1, n_mu=2, n_phi=8)
    o = dd_dlra.DDDLRA(wl)
    sub = o.subs[0]
    rng = np.random.default_rng(0)
    om = np.asarray(wl.omega_x)
    V = np.linalg.qr(o.sw_phi[:, None] * rng.standard_normal((wl.n, 5)))[0] / o.sw_phi[:, None]
    Cp = o._ip_phi(V, np.maximum(om, 0.0)[:, None] * V)
    Cm = o._ip_phi(V, np.minimum(om, 0.0)[:, None] * V)
    z = np.zeros((sub.N // sub.nxk, 5))                  # one ghost row per x-line
    worst, swapped = -np.inf, -np.inf
    for _ in range(20):
        K = rng.standard_normal((sub.N, 5))
        worst = max(worst, np.trace(o._ip_x(K, o.kstep_rhs_flux(K, Cp, Cm, z, z, sub, "x"))))
        swapped = max(swapped, np.trace(o._ip_x(K, o.kstep_rhs_flux(K, Cm, Cp, z, z, sub, "x"))))
    assert worst <= 1e-12
    assert swapped > 1e-3


def test_flux_split_rank_convergence_to_sn():
    """R21: one subdomain, RK4: with the flux split too, the error against S_N falls as
    the rank grows."""
    base = inputs.config_c0(integrator="rk4", tiles_x=1, tiles_y=1,
                            nsteps=12).with_(kstep_split="flux")
    ref = sn.scalar_flux(sn.run(base), base)
    errs = []
    for r in (5, 10, 20, 40):
        wl = base.with_(rank=r, r_aug_max=min(2 * r, base.n))
        rho = dd_dlra.DDDLRA(wl).run().scalar_flux()
        errs.append(np.linalg.norm(rho - ref) / np.linalg.norm(ref))
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[-1] < 1e-3, errs
