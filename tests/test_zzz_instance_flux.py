"""The density of one problem of a batch (dd_dlra_scalar_flux_instance) through the C ABI:
bit-identical to that problem's part of the whole batch's density, to host and to device
memory, and argument errors refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_instance_flux_is_the_problems_part_of_the_batch_density():
    import torch
    from paper_2602_14854_gb300 import binding, build, inputs
    assert torch.cuda.is_available()
    build.build()
    binding.load()
    groups = inputs.batch_problems(count=6, seed0=200, grids=(8, 16), tilings=(1, 2),
                                   directions=(16,), ranks=(2, 4), nsteps=2)
    (n, wls), = groups.items()
    s = binding.Solver(wls)
    s.step(2)
    rho = s.scalar_flux()
    for i, wl in enumerate(wls):
        part = s.instance_flux(rho, i)
        assert part.size == wl.nx * wl.ny
        assert np.array_equal(s.scalar_flux_instance(i), part)
        dev = torch.full((wl.nx * wl.ny,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        s.scalar_flux_instance(i, dev.data_ptr())
        s.sync()
        assert np.array_equal(dev.cpu().numpy(), part)
    with pytest.raises(binding.DDError):
        s.scalar_flux_instance(len(wls))
    s.close()
