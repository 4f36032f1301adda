"""Roundoff conditioning of the parity workloads (no GPU).

The projector-splitting step is sensitive to roundoff when directions with
small singular values are kept.  Rescaling the data by 1.1 changes nothing but
the rounding (every operation is homogeneous of degree one and every rank
decision is relative or uses the rescaled tolerance), so the difference of the
two rescaled oracle runs measures how much two correct FP64 implementations
can differ.  The GPU parity bar of 1e-9 is meaningful only where this is far
below it; these tests pin that for the parity workloads.
"""
import numpy as np
import pytest

from oracle import dd_dlra
from paper_2602_14854_gb300 import inputs


def rescaling_spread(wl, fac=1.1):
    a = dd_dlra.DDDLRA(wl).run()
    b = dd_dlra.DDDLRA(wl.with_(g0=wl.g0 * fac, source=wl.source * fac,
                                tol=wl.tol * fac)).run()
    ra, rb = a.scalar_flux(), b.scalar_flux() / fac
    assert a.ranks() == b.ranks()
    return np.linalg.norm(ra - rb) / np.linalg.norm(ra)


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_gaussian_32_is_well_conditioned(integrator):
    assert rescaling_spread(inputs.config_c0(integrator=integrator)) < 1e-11


def test_tolerance_workload_is_well_conditioned():
    wl = inputs.checkerboard_problem(blocks=3, cells_per_block=8, n_mu=4, n_phi=8, t_end=0.5,
                                     tol=1e-3, r_aug_max=16).with_(r_min=2, r_max=5,
                                                                   integrator="rk4")
    assert rescaling_spread(wl) < 1e-10


def test_smaller_threshold_is_ill_conditioned():
    """Keeping directions down to 1e-8 sigma_1 (explicit Euler, isotropic start)
    makes the step amplify rounding by ~1e7: the reason for tau = 1e-5."""
    wl = inputs.config_c0(nsteps=3)
    a = dd_dlra.DDDLRA(wl, tau=1e-8).run()
    b = dd_dlra.DDDLRA(wl.with_(g0=wl.g0 * 1.1), tau=1e-8).run()
    spread = np.linalg.norm(a.scalar_flux() - b.scalar_flux() / 1.1) / np.linalg.norm(a.scalar_flux())
    assert spread > 1e-9


def test_narrow_source_far_field_is_ill_conditioned():
    """A source of width 1.5 h in a corner of 4 x 4 subdomains: the far subdomains hold
    Gaussian tails (1e-160 .. 1e-300) whose rank decisions follow rounding, and 1e-15
    relative noise in the initial data moves the scalar flux by > 1e-7 after 3 steps.
    GPU results on such problems are compared against this sensitivity, not 1e-9."""
    wl = inputs.narrow_source_problem()
    a = dd_dlra.DDDLRA(wl).run(3).scalar_flux()
    rng = np.random.default_rng(3)
    b = dd_dlra.DDDLRA(wl.with_(g0=wl.g0 * (1 + 1e-15 * rng.uniform(-1, 1, wl.g0.shape)))).run(3)
    assert np.linalg.norm(b.scalar_flux() - a) / np.linalg.norm(a) > 1e-7
