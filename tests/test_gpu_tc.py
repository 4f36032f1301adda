"""The tensor-core forms (DD_TF32, DD_BF16) against the FP64 oracle, through the C ABI.

In these forms the Galerkin contractions run as tcgen05 MMAs on TMA-staged tiles (each
FP64 operand split into a high and a low TF32 / BF16 part, FP32 accumulation); the
orthonormalisations, the R factors of the QRs, the small SVDs and eigendecompositions and
the advection K-step stay FP64.  Bounds: 1e-5 (TF32) and 1e-3 (BF16) on the scalar flux,
except where a test states the problem's own sensitivity.
"""
import os

import numpy as np
import pytest

from oracle import dd_dlra

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
BOUND = {"tf32": 1e-5, "bf16": 1e-3}


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


def run_tc(B, wl, prec, nsteps=None, graph=True):
    s = B.Solver(wl, precision=prec, use_graph=graph)
    s.step(wl.nsteps if nsteps is None else nsteps)
    rho = s.scalar_flux()
    ranks = list(s.ranks()[0])
    prof = s.profile(1)
    s.close()
    return rho, ranks, prof


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_small_random_problem(B, prec, integrator):
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(0, nx=8, ny=8, n_mu=2, n_phi=8, rank=3, r_aug_max=6,
                                     integrator=integrator, nsteps=3)
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, prof = run_tc(B, wl, prec)
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < BOUND[prec]
    # the tensor-core kernels ran (every step: both kernels, several launches)
    assert prof["k_tc_tall"][1] > 0 and prof["k_tc_gram"][1] > 0


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_ragged_tiling_odd_capacity(B, prec):
    """3/5/8-cell columns, 5/5 rows; r_aug_max = 7 gives an odd column capacity, rounded up
    to an even one in these forms (TMA rows on 16-byte boundaries)."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(3, nx=16, ny=10, n_mu=2, n_phi=8, rank=3, r_aug_max=7,
                                     integrator="rk4", nsteps=3, xcuts=[0, 3, 8, 16],
                                     ycuts=[0, 5, 10])
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, _ = run_tc(B, wl, prec)
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < BOUND[prec]


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_flux_split_form(B, prec):
    """The flux-split K-step (eight angular blocks, C+ and C- among them, on the tensor cores)."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(1, nx=8, ny=8, n_mu=2, n_phi=8, rank=3, r_aug_max=6,
                                     integrator="rk4", nsteps=3).with_(kstep_split="flux")
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, _ = run_tc(B, wl, prec)
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < BOUND[prec]


def test_inflow_problem(B):
    """Physical inflow: the angular coefficients stay FP64 (the inflow sides enter them as
    one-row neighbours); the other contractions run on the tensor cores."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(5, nx=12, ny=12, tiles_x=3, tiles_y=3, n_mu=2, n_phi=8,
                                     rank=3, r_aug_max=8, integrator="rk4", nsteps=3)
    wl = wl.with_(inflow={"x_lo": (np.linspace(0.5, 1.5, 12), np.linspace(0.1, 1.0, wl.n))})
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, prof = run_tc(B, wl, "tf32")
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < 1e-5
    assert prof["k_ang_coeffs"][1] > 0


def test_pointsource_full_size(B):
    """The point-source workload (128^2, 4x4, 512 directions, rank 10, RK4), all 86 steps, in
    graph replay, against the stored oracle result.  The FP32-level error of the tall
    products (the truncation's rotations, K0 = X (S <V, V_hat>)), ~1e-7 relative per product
    and phase, adds up linearly over the 86 steps: measured 6.6e-5 (TF32); held to 1e-4 and,
    for BF16, to 1e-3."""
    from paper_2602_14854_gb300 import inputs
    gold = np.load(os.path.join(HERE, "golden", "pointsource_128_rk4_t1.npz"))
    wl = inputs.config_c1()
    for prec, bound in (("tf32", 1e-4), ("bf16", 1e-3)):
        rho, ranks, _ = run_tc(B, wl, prec)
        assert ranks == list(gold["ranks"])
        assert rel(rho, gold["rho"]) < bound, prec


def test_lognormal_full_size(B):
    """The lognormal medium at full size (512^2, 8x8, 2048 directions, rank 20), 1 step."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.lognormal_problem(nsteps=1)
    ref = dd_dlra.DDDLRA(wl).run()
    for prec in ("tf32", "bf16"):
        rho, ranks, _ = run_tc(B, wl, prec)
        assert ranks == ref.ranks()
        assert rel(rho, ref.scalar_flux()) < BOUND[prec], prec


def test_small_gaussian_euler(B):
    """The small Gaussian (32^2, 2x2, 128 directions, rank 5, 50 explicit Euler steps): the
    FP32-level error of the contractions accumulates over the 50 steps to ~3e-5 (TF32) and
    ~1e-4 (BF16); held to 1e-4 and 1e-3."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.config_c0()
    ref = dd_dlra.DDDLRA(wl).run()
    for prec, bound in (("tf32", 1e-4), ("bf16", 1e-3)):
        rho, ranks, _ = run_tc(B, wl, prec)
        assert ranks == ref.ranks()
        assert rel(rho, ref.scalar_flux()) < bound, prec


def run_products(B, wl, products, nsteps=None, precision="fp64"):
    s = B.Solver(wl, products=products, use_graph=True, precision=precision)
    s.step(wl.nsteps if nsteps is None else nsteps)
    rho = s.scalar_flux()
    ranks = list(s.ranks()[0])
    prof = s.profile(1)
    s.close()
    return rho, ranks, prof


@pytest.mark.parametrize("seed,cuts", [(0, None), (3, ([0, 3, 8, 16], [0, 5, 10]))])
def test_ozaki_products_small(B, seed, cuts):
    """FP64 tall products on the BF16 tensor cores (Ozaki splitting): FP64-level error, so
    the FP64 bound 1e-9 holds; ragged 3/5/8-cell tiles and an odd column capacity included."""
    from paper_2602_14854_gb300 import inputs
    kw = {} if cuts is None else {"nx": 16, "ny": 10, "xcuts": cuts[0], "ycuts": cuts[1]}
    wl = inputs.random_small_problem(seed, **{"nx": 8, "ny": 8, **kw}, n_mu=2, n_phi=8, rank=3,
                                     r_aug_max=7, integrator="rk4", nsteps=3)
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, prof = run_products(B, wl, "tensor")
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < 1e-9
    # the tall products and the orthonormalisations' Grams
    assert prof["k_oz_tall"][1] > 0 and prof["k_oz_gram"][1] > 0


@pytest.mark.parametrize("seed,cuts", [(1, None), (4, ([0, 3, 8, 16], [0, 5, 10]))])
def test_ozaki_lstep_products_euler(B, seed, cuts):
    """Explicit Euler with the Ozaki products: the advection L-step runs as three products
    over the direction rows (with S2^T, W_+^T = (A_+ S2 - G_lo)^T, W_-^T = (A_- S2 + G_hi)^T),
    the last two accumulated row by row with the scales dt kappa_q of their upwind side, not
    as k_lstep_adv; FP64 bound 1e-9 and identical ranks on even and ragged tilings."""
    from paper_2602_14854_gb300 import inputs
    kw = {} if cuts is None else {"nx": 16, "ny": 10, "xcuts": cuts[0], "ycuts": cuts[1]}
    wl = inputs.random_small_problem(seed, **{"nx": 8, "ny": 8, **kw}, n_mu=2, n_phi=8, rank=3,
                                     r_aug_max=7, integrator="euler", nsteps=4)
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, prof = run_products(B, wl, "tensor")
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < 1e-9
    assert prof["k_lstep_prod"][1] > 0 and "k_lstep_adv" not in prof


@pytest.mark.parametrize("prec", ["tf32", "bf16", "mixed"])
def test_ozaki_lstep_products_reduced_forms(B, prec):
    """The reduced-precision forms with the Ozaki products take the same FP64-accurate
    product L-step (in place of their FP32 stages) and stay within their bounds."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(2, nx=16, ny=10, xcuts=[0, 3, 8, 16], ycuts=[0, 5, 10],
                                     n_mu=2, n_phi=8, rank=3, r_aug_max=7, integrator="euler",
                                     nsteps=4)
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, prof = run_products(B, wl, "tensor", precision=prec)
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < BOUND.get(prec, 1e-5)
    assert prof["k_lstep_prod"][1] > 0 and "k_lstep_adv" not in prof


def test_ozaki_products_inflow(B):
    """Ozaki products with a physical inflow side (the inflow column in the augmentation's L0,
    neighbour blocks absent on the boundary) and explicit Euler; FP64 bound 1e-9."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.random_small_problem(5, nx=12, ny=12, tiles_x=3, tiles_y=3, n_mu=2, n_phi=8,
                                     rank=3, r_aug_max=8, integrator="euler", nsteps=3)
    wl = wl.with_(inflow={"x_lo": (np.linspace(0.5, 1.5, 12), np.linspace(0.1, 1.0, wl.n))})
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, prof = run_products(B, wl, "tensor")
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < 1e-9
    assert prof["k_oz_tall"][1] > 0


def test_ozaki_products_pointsource(B):
    """The point-source workload, all 86 steps, Ozaki products: within 1e-9 of the stored
    oracle result (measured 1.7e-12, as the FP64 CUDA-core products)."""
    from paper_2602_14854_gb300 import inputs
    gold = np.load(os.path.join(HERE, "golden", "pointsource_128_rk4_t1.npz"))
    wl = inputs.config_c1()
    rho, ranks, _ = run_products(B, wl, "tensor")
    assert ranks == list(gold["ranks"])
    assert rel(rho, gold["rho"]) < 1e-9


def test_ozaki_products_lognormal(B):
    """The lognormal medium at full size, 1 step, Ozaki products, against the oracle."""
    from paper_2602_14854_gb300 import inputs
    wl = inputs.lognormal_problem(nsteps=1)
    ref = dd_dlra.DDDLRA(wl).run()
    rho, ranks, _ = run_products(B, wl, "tensor")
    assert ranks == ref.ranks()
    assert rel(rho, ref.scalar_flux()) < 1e-9
