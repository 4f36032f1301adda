"""Solver memory from the caller's allocator (dd_set_allocator) through the C ABI: every
device buffer of a solver comes from PyTorch's caching allocator and goes back to it at
destroy, and the results are bit-identical to those of a solver on cudaMalloc memory."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_solver_memory_from_the_torch_allocator():
    import torch
    from paper_2602_14854_gb300 import binding, build, inputs
    assert torch.cuda.is_available()
    build.build()
    binding.load()
    wl = inputs.config_c0(nsteps=3)
    ref = binding.Solver(wl)
    ref.step(3)
    rho_ref = ref.scalar_flux()
    ref.close()

    live, calls = {}, {"alloc": 0, "release": 0}

    def alloc(nbytes):
        p = torch.cuda.caching_allocator_alloc(nbytes)
        calls["alloc"] += 1
        live[p] = nbytes
        return p

    def release(p):
        calls["release"] += 1
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    binding.set_allocator(alloc, release)
    try:
        s = binding.Solver(wl)
    finally:
        binding.set_allocator()
    assert calls["alloc"] >= 30
    assert torch.cuda.memory_allocated() - before >= sum(live.values())
    s.step(3)
    rho = s.scalar_flux()
    s.close()
    assert calls["release"] == calls["alloc"] and not live
    assert np.array_equal(rho, rho_ref)
