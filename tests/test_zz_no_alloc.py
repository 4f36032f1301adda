"""The allocation-free density readout (dd_dlra_scalar_flux_noalloc) against the
regular one (dd_dlra_scalar_flux), through the C ABI.

The allocation-free call serves callers that must not allocate device memory
when they read the density (e.g. under an allocate-at-start-up-only policy); it
keeps its scratch in a fixed device array instead of solver workspace.  This file
is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-9     # the parity tolerance of the GPU tests (rel-L2)


@pytest.fixture(scope="module")
def B():
    import torch
    from paper_2602_14854_gb300 import binding, build
    assert torch.cuda.is_available()
    build.build()
    binding.load()
    return binding


def test_noalloc_flux_matches_regular_readout(B):
    import torch
    from paper_2602_14854_gb300 import inputs
    wl = inputs.config_c0(nsteps=4)
    s = B.Solver(wl)
    out = torch.empty(wl.ncells, dtype=torch.float64, device="cuda")
    for call, nsteps in enumerate((3, 1)):          # two calls in a row, state changing between
        s.step(nsteps)
        ref = s.scalar_flux()
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        s.scalar_flux_noalloc(out.data_ptr())
        s.sync()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), call
    s.close()


def test_noalloc_flux_rejects_oversized_solver(B):
    """17 x 17 subdomains with rank capacity 63 need more scratch than the fixed
    16384 doubles: the call refuses with DD_ERR_ARG."""
    import torch
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(1, nx=68, ny=68, tiles_x=17, tiles_y=17, n_mu=2, n_phi=32,
                                     rank=21, r_aug_max=21, nsteps=1)
    s = B.Solver(wl)
    out = torch.empty(wl.ncells, dtype=torch.float64, device="cuda")
    with pytest.raises(B.DDError) as e:
        s.scalar_flux_noalloc(out.data_ptr())
    assert e.value.status == 1 and "exceeds" in str(e.value)
    s.close()


def test_noalloc_flux_is_capturable_on_the_solvers_stream(B):
    """A solver created on a user stream: after one ordinary call, the readout is
    captured on that stream in global capture mode (which refuses allocation and
    synchronisation inside the capture), and replaying the graph reproduces the
    regular readout of the state current at replay time."""
    import torch
    from paper_2602_14854_gb300 import inputs
    wl = inputs.config_c0(nsteps=4)
    st = torch.cuda.Stream()
    s = B.Solver(wl, stream=st.cuda_stream)
    out = torch.empty(wl.ncells, dtype=torch.float64, device="cuda")
    s.step(2)
    s.scalar_flux_noalloc(out.data_ptr())            # warm-up, outside any capture
    s.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st, capture_error_mode="global"):
        s.scalar_flux_noalloc(out.data_ptr())
    s.step(1)
    s.sync()
    ref = s.scalar_flux()
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)
    del g
    s.close()
