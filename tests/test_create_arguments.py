"""The create call's argument checks through the C ABI, on the CPU: each inconsistent
problem or option is refused with DD_ERR_ARG and its message before any device memory is
allocated (the checks run before the first CUDA allocation)."""
import numpy as np
import pytest

from paper_2602_14854_gb300 import binding, build, inputs


@pytest.fixture(scope="module")
def B():
    build.build()
    binding.load()
    return binding


def base(**kw):
    return inputs.random_small_problem(3, nx=8, ny=8, tiles_x=2, tiles_y=2, n_mu=2, n_phi=8,
                                       rank=2, r_aug_max=4, nsteps=1, **kw)


CASES = [
    ("r_aug_max above the column capacity", dict(r_aug_max=65), "r_aug_max must be in"),
    ("stored rank above r_aug_max", dict(rank=5), "stored-rank cap must be in"),
    ("augmentation input wider than 64", dict(rank=22, r_aug_max=64), "3 * stored-rank cap"),
    ("fewer directions than 3 r", dict(rank=6, r_aug_max=12), "directions"),
    ("tiling not ending at nx", dict(xcuts=[0, 4, 7]), "tiling cuts"),
    ("tiling not increasing", dict(xcuts=[0, 4, 4, 8]), "not increasing"),
    ("non-positive time step", dict(dt=0.0), "dt / tau"),
    ("non-positive quadrature weight", "w0", "weights must be positive"),
    ("unknown integrator", dict(integrator="midpoint"), None),
]


@pytest.mark.parametrize("name,change,msg", CASES, ids=[c[0] for c in CASES])
def test_create_refuses(B, name, change, msg):
    wl = base()
    if change == "w0":
        w = wl.w.copy()
        w[3] = 0.0
        wl = wl.with_(w=w)
    elif "integrator" in change:
        with pytest.raises(ValueError):             # the binding knows only euler / rk4
            B.Solver(wl.with_(**change))
        return
    else:
        wl = wl.with_(**change)
    with pytest.raises(B.DDError) as e:
        B.Solver(wl)
    assert e.value.status == 1, str(e.value)
    assert msg in str(e.value), str(e.value)


def test_batch_with_different_integrators_is_refused(B):
    a = base()
    with pytest.raises(B.DDError) as e:
        B.Solver([a, a.with_(integrator="rk4")])
    assert e.value.status == 1 and "share" in str(e.value)
