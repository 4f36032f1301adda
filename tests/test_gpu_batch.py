"""Batched form: independent problems sharing a direction table advance in the same
launches (dd_dlra_create_batch); every problem must match the oracle run on its own
(rel-L2 <= 1e-9) and the same problem run alone on the GPU."""
import numpy as np
import pytest

from oracle import dd_dlra
from paper_2602_14854_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def test_batch_matches_oracle_and_single(B):
    groups = inputs.batch_problems(count=8, seed0=100, grids=(8, 16), tilings=(1, 2),
                                   directions=(16, 32), ranks=(2, 4), nsteps=3)
    assert sum(len(v) for v in groups.values()) == 8
    for n, wls in groups.items():
        s = B.Solver(wls, use_graph=True)
        s.step(3)
        rho = s.scalar_flux()
        for i, wl in enumerate(wls):
            ref = dd_dlra.DDDLRA(wl).run(3).scalar_flux()
            got = s.instance_flux(rho, i)
            assert rel(got, ref) < 1e-9, (wl.name, rel(got, ref))
            one = B.Solver(wl)
            one.step(3)
            assert rel(got, one.scalar_flux()) < 1e-12
            one.close()
        s.close()


def test_batch_rejects_mismatched_options(B):
    a = inputs.random_small_problem(1, nx=8, ny=8, n_mu=2, n_phi=8, rank=2, r_aug_max=4)
    b = a.with_(integrator="rk4")
    with pytest.raises(B.DDError):
        B.Solver([a, b])


def test_solvers_of_different_width_coexist(B):
    """Kernel attributes are per process: a wide solver (stored rank 12) created before a
    narrow one (rank 2) must still step correctly after the narrow one exists."""
    wide = inputs.random_small_problem(11, nx=16, ny=16, n_mu=4, n_phi=16, rank=12,
                                       r_aug_max=24, integrator="rk4", nsteps=3)
    narrow = inputs.random_small_problem(12, nx=8, ny=8, n_mu=2, n_phi=8, rank=2, r_aug_max=4,
                                         integrator="rk4", nsteps=3)
    sw = B.Solver(wide, use_graph=True)
    sn = B.Solver(narrow, use_graph=True)
    sn.step(3)
    sw.step(3)
    assert rel(sw.scalar_flux(), dd_dlra.DDDLRA(wide).run(3).scalar_flux()) < 1e-9
    assert rel(sn.scalar_flux(), dd_dlra.DDDLRA(narrow).run(3).scalar_flux()) < 1e-9
    sw.close()
    sn.close()
