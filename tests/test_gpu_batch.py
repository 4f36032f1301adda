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


def test_full_size_batch_sampled_against_oracle(B):
    """The 64-problem batch at full size (64^2/128^2/256^2 grids, 2x2/4x4 tilings,
    128/512/1024 directions, ranks 4..21, RK4) in the benchmark's launch configuration:
    one graph-replayed solver per direction group, 2 steps.  Three problems, sampled, are
    checked against the oracle run on each alone: the 256^2, 2x2, rank-21 Gaussian (128-cell
    lines at r_t up to 42, beyond the eigenbasis K-step's tile: the FP64 matrix stencil
    takes them, in the mixed form too), a 512- and a 1024-direction narrow point source."""
    groups = sorted(inputs.batch_problems(count=64, nsteps=2).items())
    sample = ("batch8-", "batch19-", "batch1-")
    checked = 0
    for n, wls in groups:
        picks = [(i, wl) for i, wl in enumerate(wls) if wl.name.startswith(sample)]
        if not picks:
            continue
        s = B.Solver(wls, use_graph=True)
        s.step(2)
        rho = s.scalar_flux()
        got = {i: s.instance_flux(rho, i) for i, _ in picks}
        s.close()
        got_mixed = {}
        if any(wl.name.startswith("batch8-") for _, wl in picks):
            m = B.Solver(wls, use_graph=True, precision="mixed")
            m.step(2)
            rm = m.scalar_flux()
            got_mixed = {i: m.instance_flux(rm, i) for i, wl in picks if wl.name.startswith("batch8-")}
            m.close()
        for i, wl in picks:
            ref = dd_dlra.DDDLRA(wl).run(2).scalar_flux()
            assert rel(got[i], ref) < 1e-9, (wl.name, rel(got[i], ref))
            if i in got_mixed:
                assert rel(got_mixed[i], ref) < 1e-5, (wl.name, rel(got_mixed[i], ref))
            checked += 1
    assert checked == 3
