"""Mixed-precision form (DD_MIXED) against the FP64 CPU oracle.

FP32 arithmetic for the stencil and the increments of the K-/L-/collision-step ODEs;
FP64 for the updates, the orthonormalisations, the small eigen/SVD problems and
reductions.
Target: scalar-flux rel-L2 <= 1e-5 against the oracle (FP32 target of the task
statement), on the same workloads as the FP64 parity tests.
"""
import os

import numpy as np
import pytest

from oracle import dd_dlra
from paper_2602_14854_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-5
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def B():
    import torch
    from paper_2602_14854_gb300 import binding, build
    assert torch.cuda.is_available()
    build.build()
    binding.load()
    return binding


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_mixed_gaussian_32(B, integrator):
    wl = inputs.config_c0(integrator=integrator)
    s = B.Solver(wl, precision="mixed")
    s.step(wl.nsteps)
    ref = dd_dlra.DDDLRA(wl).run().scalar_flux()
    assert rel(s.scalar_flux(), ref) < TOL_MIXED
    s.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_mixed_small_random(B, seed):
    wl = inputs.random_small_problem(seed, nx=8, ny=8, n_mu=2, n_phi=8, rank=3, r_aug_max=6,
                                     integrator="rk4", nsteps=4)
    s = B.Solver(wl, precision="mixed")
    s.step(wl.nsteps)
    ref = dd_dlra.DDDLRA(wl).run().scalar_flux()
    assert rel(s.scalar_flux(), ref) < TOL_MIXED
    s.close()


def test_mixed_pointsource_full_size(B):
    gold = np.load(os.path.join(HERE, "golden", "pointsource_128_rk4_t1.npz"))
    wl = inputs.config_c1()
    s = B.Solver(wl, use_graph=True, precision="mixed")
    s.step(wl.nsteps)
    assert rel(s.scalar_flux(), gold["rho"]) < TOL_MIXED
    s.close()
