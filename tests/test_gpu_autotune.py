"""The autotuner (dd_options.autotune) and the per-family choice of the FP64 tall-product
engine (dd_options.products = DD_PRODUCTS_AUTO), through the C ABI.

Whatever the autotuner picks (the FP64 CUDA-core or the tensor-core Ozaki products per row
family, the Gram chunk counts), the arithmetic stays FP64-accurate: the FP64 bound 1e-9
against the oracle holds with the stored ranks identical.
"""
import os

import numpy as np
import pytest

from oracle import dd_dlra

pytestmark = pytest.mark.gpu

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


def test_autotuned_small_problem_matches_oracle(B):
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(2, nx=16, ny=16, n_mu=2, n_phi=8, rank=3, r_aug_max=8,
                                     integrator="rk4", nsteps=3)
    ref = dd_dlra.DDDLRA(wl).run()
    s = B.Solver(wl, products="auto", autotune=True, use_graph=True)
    choice, ms = s.tuning()
    s.step(wl.nsteps)
    rho, ranks = s.scalar_flux(), list(s.ranks()[0])
    s.close()
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < 1e-9
    # both engines and the chunk candidates were timed for both row families
    assert all(t > 0 for t in ms), ms
    assert choice["oz_spatial"] in (0, 1) and choice["oz_angular"] in (0, 1)
    assert choice["chunks_spatial"] >= 1 and choice["chunks_angular"] >= 1


def test_choices_are_cached_per_shape(B):
    """A second solver of the same shape takes the cached choices (same timings, no new
    trial); a solver with autotune off reports no timings."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(4, nx=16, ny=16, n_mu=2, n_phi=8, rank=3, r_aug_max=8,
                                     integrator="euler", nsteps=2)
    a = B.Solver(wl, products="auto", autotune=True)
    b = B.Solver(wl, products="auto", autotune=True)
    c = B.Solver(wl, products="auto")
    ta, tb, tc = a.tuning(), b.tuning(), c.tuning()
    for s in (a, b, c):
        s.close()
    assert ta == tb
    assert all(t == -1.0 for t in tc[1])


def test_forced_choices_are_kept(B):
    """products = fp64 / tensor fix the engine: the autotuner times only the chunk counts."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(6, nx=16, ny=16, n_mu=2, n_phi=8, rank=3, r_aug_max=8,
                                     integrator="euler", nsteps=2)
    for prod, flag in (("fp64", 0), ("tensor", 1)):
        s = B.Solver(wl, products=prod, autotune=True)
        choice, ms = s.tuning()
        s.close()
        assert choice["oz_spatial"] == flag and choice["oz_angular"] == flag
        assert ms[0] == ms[1] == ms[4] == ms[5] == -1.0
        assert ms[2] > 0 and ms[6] > 0


def test_autotuned_pointsource_full_run(B):
    """The point-source workload, all 86 steps, autotuned: within 1e-9 of the stored oracle
    result, stored ranks identical."""
    from paper_2602_14854_gb300 import inputs
    gold = np.load(os.path.join(HERE, "golden", "pointsource_128_rk4_t1.npz"))
    wl = inputs.config_c1()
    s = B.Solver(wl, products="auto", autotune=True, use_graph=True)
    s.step(wl.nsteps)
    rho, ranks = s.scalar_flux(), list(s.ranks()[0])
    s.close()
    assert ranks == list(gold["ranks"])
    assert rel(rho, gold["rho"]) < 1e-9


def test_autotuned_lognormal_prefix(B):
    """The lognormal medium at full size, autotuned (the tensor-core products win there):
    20 steps against the stored oracle result on 16384 sampled cells and the whole norm."""
    from paper_2602_14854_gb300 import inputs
    gold = np.load(os.path.join(HERE, "golden", "lognormal_512_prefix20.npz"))
    wl = inputs.lognormal_problem()
    s = B.Solver(wl, products="auto", autotune=True, use_graph=True)
    choice, _ = s.tuning()
    s.step(int(gold["nsteps"]))
    rho, ranks = s.scalar_flux(), list(s.ranks()[0])
    s.close()
    assert choice["oz_spatial"] == 1
    assert ranks == list(gold["ranks"])
    assert rel(rho[gold["idx"]], gold["rho"]) < 1e-9
    assert abs(np.linalg.norm(rho) - float(gold["norm"])) < 1e-9 * float(gold["norm"])
