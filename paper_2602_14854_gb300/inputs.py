"""Seeded synthetic problem data for the DD-DLRA time step.

This module only builds *problem data*: the grid, the subdomain tiling, the
discrete-ordinates direction table, the material fields (sigma_s, sigma_a, Q)
and the isotropic initial density g(x, y).  It contains none of the method's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs from
it.

Problem family (Section 2, Eq. (rt)): 2D space x angle radiative transfer,
    d_t f + c_adv Omega . grad f = sigma_s/|S| rho - sigma_t f + Q,
    sigma_t = sigma_s + sigma_a,  rho = sum_q w_q f_q.
The paper's own angular model is the circle (phi only, |S| = 2*pi,
Omega = (cos phi, sin phi), equidistant phi).  The workloads below use the
product set of Gauss-Legendre mu levels times equidistant phi, projected onto
the plane: Omega = (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi),
w = w_mu * 2*pi / n_phi, |S| = 4*pi.  ``n_mu = 0`` selects the paper's circle.

Cells are numbered x-fastest over the global grid: c = j * nx + i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    xcuts: list          # cell indices of the subdomain interfaces in x, [0, ..., nx]
    ycuts: list          # same in y, [0, ..., ny]
    omega_x: np.ndarray  # (n,)
    omega_y: np.ndarray  # (n,)
    w: np.ndarray        # (n,) quadrature weights, sum = |S|
    sigma_s: np.ndarray  # (ny*nx,)
    sigma_a: np.ndarray  # (ny*nx,)
    source: np.ndarray   # (ny*nx,) isotropic source Q
    g0: np.ndarray       # (ny*nx,) isotropic initial data f(0, x, y, Omega) = g0(x, y)
    dt: float
    nsteps: int
    rank_mode: str = "fixed"   # "fixed" or "tol"
    rank: int = 5              # fixed-rank mode: stored rank r
    tol: float = 0.0           # tolerance mode: absolute truncation tolerance
    r_min: int = 1             # tolerance mode: stored-rank floor
    r_max: int = 64            # tolerance mode: stored-rank ceiling
    r_aug_max: int = 10        # cap on the intermediate (augmented) rank r_t
    integrator: str = "euler"  # "euler" or "rk4"
    c_adv: float = 1.0
    n_mu: int = 0              # polar levels of the direction table (0: the paper's circle)
    n_phi: int = 0             # azimuths per level
    mass_fix: bool = False     # conserved-moment correction at the end of every step
    splitting: str = "lie"     # "lie" (x, y, collision) or "strang" (x/2, y/2, collision, y/2, x/2)
    kstep_split: str = "eigen" # C+/C- of the advection K-step: "eigen" (Appendix A) or "flux"
    # physical inflow f(s, Omega) = g(s) h(Omega) on a side ("x_lo", "x_hi", "y_lo", "y_hi")
    # for the directions entering through it: side -> (g over the side's cells, h over the
    # directions); absent sides have zero inflow
    inflow: dict = field(default_factory=dict)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.w.shape[0])

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    @property
    def ncells(self) -> int:
        return self.nx * self.ny

    @property
    def nsub(self) -> int:
        return (len(self.xcuts) - 1) * (len(self.ycuts) - 1)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def product_quadrature(n_mu: int, n_phi: int):
    """Direction table (Omega_x, Omega_y, w).

    n_mu > 0: Gauss-Legendre mu levels x equidistant phi_j = (j + 1/2) 2 pi / n_phi,
    projected on the plane; sum w = 4 pi.
    n_mu = 0: the paper's circle, Omega = (cos phi, sin phi), w = 2 pi / n_phi; sum w = 2 pi.
    Directions are ordered mu-major, phi-minor.
    """
    phi = (np.arange(n_phi) + 0.5) * (2.0 * math.pi / n_phi)
    if n_mu == 0:
        return np.cos(phi), np.sin(phi), np.full(n_phi, 2.0 * math.pi / n_phi)
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    s = np.sqrt(1.0 - mu * mu)
    ox = (s[:, None] * np.cos(phi)[None, :]).reshape(-1)
    oy = (s[:, None] * np.sin(phi)[None, :]).reshape(-1)
    w = (wmu[:, None] * np.full(n_phi, 2.0 * math.pi / n_phi)[None, :]).reshape(-1)
    return ox, oy, w


def _cell_centres(nx, ny, x0, x1, y0, y1):
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * hx
    yc = y0 + (np.arange(ny) + 0.5) * hy
    X, Y = np.meshgrid(xc, yc)          # (ny, nx), x fastest
    return X.reshape(-1), Y.reshape(-1)


def uniform_cuts(ncell: int, nparts: int):
    assert ncell % nparts == 0
    b = ncell // nparts
    return [i * b for i in range(nparts + 1)]


def gaussian_problem(*, name, nx, ny, x0, x1, y0, y1, tiles_x, tiles_y, n_mu, n_phi,
                     centre, width, sigma_s=1.0, sigma_a=0.0, rank=5, r_aug_max=None,
                     t_end=None, nsteps=None, cfl=0.5, integrator="euler", xcuts=None,
                     ycuts=None) -> Workload:
    """Homogeneous medium, isotropic Gaussian initial data, zero inflow.

    dt = cfl * h; with ``t_end`` the step count is ceil(t_end / (cfl*h)) and dt is
    shrunk to land on t_end exactly.
    """
    ox, oy, w = product_quadrature(n_mu, n_phi)
    X, Y = _cell_centres(nx, ny, x0, x1, y0, y1)
    g0 = np.exp(-((X - centre[0]) ** 2 + (Y - centre[1]) ** 2) / (2.0 * width * width))
    h = min((x1 - x0) / nx, (y1 - y0) / ny)
    if t_end is not None:
        nsteps = int(math.ceil(t_end / (cfl * h) - 1e-12))
        dt = t_end / nsteps
    else:
        dt = cfl * h
    ncell = nx * ny
    return Workload(
        name=name, nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1,
        xcuts=list(xcuts) if xcuts is not None else uniform_cuts(nx, tiles_x),
        ycuts=list(ycuts) if ycuts is not None else uniform_cuts(ny, tiles_y),
        omega_x=ox, omega_y=oy, w=w,
        sigma_s=np.full(ncell, float(sigma_s)), sigma_a=np.full(ncell, float(sigma_a)),
        source=np.zeros(ncell), g0=g0, dt=dt, nsteps=int(nsteps),
        rank_mode="fixed", rank=rank,
        r_aug_max=(2 * rank if r_aug_max is None else r_aug_max),
        integrator=integrator, n_mu=n_mu, n_phi=n_phi,
    )


def config_c0(**kw) -> Workload:
    """Plain FP64 DD-DLRA small case: [0,1]^2, 32x32 cells, 2x2 subdomains of 16x16,
    128 directions (8 Gauss-Legendre mu x 16 phi), rank 5, sigma_s=1, sigma_a=0, Q=0,
    isotropic Gaussian exp(-|x-0.5|^2 / (2*0.05^2)), zero inflow, explicit Euler,
    dt = 0.5 h, 50 steps."""
    args = dict(name="gaussian-32x32-2x2-n128-r5", nx=32, ny=32, x0=0.0, x1=1.0, y0=0.0,
                y1=1.0, tiles_x=2, tiles_y=2, n_mu=8, n_phi=16, centre=(0.5, 0.5),
                width=0.05, rank=5, nsteps=50)
    args.update(kw)
    return gaussian_problem(**args)


def config_c1(**kw) -> Workload:
    """Point-source case: [-1.5,1.5]^2, 128x128 cells, 4x4 subdomains of 32x32,
    512 directions (16 mu x 32 phi), rank 10, sigma_s=1, sigma_a=0, isotropic
    Gaussian of width 0.03 at the origin, zero inflow, dt = 0.5 h up to t = 1
    (86 steps).  Every sub-step ODE is integrated with classic RK4, the paper's
    integrator (with explicit Euler the projector-splitting S- and L-steps leave
    an O((c dt/h)^2) error per step at Courant number 0.5)."""
    args = dict(name="pointsource-128x128-4x4-n512-r10", nx=128, ny=128, x0=-1.5, x1=1.5,
                y0=-1.5, y1=1.5, tiles_x=4, tiles_y=4, n_mu=16, n_phi=32,
                centre=(0.0, 0.0), width=0.03, rank=10, t_end=1.0, integrator="rk4")
    args.update(kw)
    return gaussian_problem(**args)


def checkerboard_problem(**kw) -> Workload:
    """Heterogeneous thick/thin medium: [0,7]^2 as 7x7 unit blocks, 224x224 cells,
    49 block-aligned subdomains.  Absorber blocks ((I+J) odd): sigma_a=10, sigma_s=0;
    other blocks sigma_s=1, sigma_a=0; isotropic Q=1 in the centre block (3,3).
    1024 directions (16 mu x 64 phi), tolerance-adaptive ranks 4..21 (tol 1e-4; the
    stated 4..30 is capped at 21 so that the augmentation input, 3 r columns, fits the
    64-column capacity), r_t <= 42, t = 3.2.  The initial state is the paper's small
    constant 1e-9."""
    nb = kw.pop("blocks", 7)
    cells_per_block = kw.pop("cells_per_block", 32)
    n_mu = kw.pop("n_mu", 16)
    n_phi = kw.pop("n_phi", 64)
    t_end = kw.pop("t_end", 3.2)
    nx = ny = nb * cells_per_block
    ox, oy, w = product_quadrature(n_mu, n_phi)
    X, Y = _cell_centres(nx, ny, 0.0, float(nb), 0.0, float(nb))
    I = np.minimum(np.floor(X).astype(int), nb - 1)
    J = np.minimum(np.floor(Y).astype(int), nb - 1)
    absorber = ((I + J) % 2) == 1
    sig_s = np.where(absorber, 0.0, 1.0)
    sig_a = np.where(absorber, 10.0, 0.0)
    src = np.where((I == nb // 2) & (J == nb // 2), 1.0, 0.0)
    h = 1.0 / cells_per_block
    nsteps = int(math.ceil(t_end / (0.5 * h) - 1e-12))
    wl = Workload(
        name=f"checkerboard-{nx}x{ny}-{nb}x{nb}-n{ox.shape[0]}-tol",
        nx=nx, ny=ny, x0=0.0, x1=float(nb), y0=0.0, y1=float(nb),
        xcuts=uniform_cuts(nx, nb), ycuts=uniform_cuts(ny, nb),
        omega_x=ox, omega_y=oy, w=w, sigma_s=sig_s, sigma_a=sig_a, source=src,
        g0=np.full(nx * ny, 1e-9), dt=t_end / nsteps, nsteps=nsteps,
        rank_mode="tol", rank=4, tol=kw.pop("tol", 1e-4), r_min=4, r_max=kw.pop("r_max", 21),
        r_aug_max=kw.pop("r_aug_max", 42), n_mu=n_mu, n_phi=n_phi,
    )
    return wl.with_(**kw) if kw else wl


def hohlraum_problem(**kw) -> Workload:
    """Hohlraum-type inflow problem: [0,1]^2, 128x128 cells, 4x4 subdomains, 512
    directions (16 mu x 32 phi); radiation enters through x = 0 with f = 1 for
    Omega_x >= 0 (the inflow of Section 4's Hohlraum test), zero inflow elsewhere;
    vacuum except one absorbing block (sigma_a = 10) in the centre [0.4,0.6]^2, standing
    in for the paper's block layout, which is given only as a figure; initial state
    1e-9; tolerance-adaptive ranks (tol 1e-3, the paper's value for the domain
    decomposition run), ranks 2..16, r_t <= 32; dt = h/2 up to t = 0.5."""
    n_mu = kw.pop("n_mu", 16)
    n_phi = kw.pop("n_phi", 32)
    nx = ny = kw.pop("cells", 128)
    tiles = kw.pop("tiles", 4)
    t_end = kw.pop("t_end", 0.5)
    ox, oy, w = product_quadrature(n_mu, n_phi)
    X, Y = _cell_centres(nx, ny, 0.0, 1.0, 0.0, 1.0)
    block = (np.abs(X - 0.5) < 0.1) & (np.abs(Y - 0.5) < 0.1)
    h = 1.0 / nx
    nsteps = int(math.ceil(t_end / (0.5 * h) - 1e-12))
    wl = Workload(
        name=f"hohlraum-{nx}x{ny}-{tiles}x{tiles}-n{ox.shape[0]}-tol",
        nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0,
        xcuts=uniform_cuts(nx, tiles), ycuts=uniform_cuts(ny, tiles),
        omega_x=ox, omega_y=oy, w=w, sigma_s=np.zeros(nx * ny),
        sigma_a=np.where(block, 10.0, 0.0), source=np.zeros(nx * ny),
        g0=np.full(nx * ny, 1e-9), dt=t_end / nsteps, nsteps=nsteps,
        rank_mode="tol", rank=2, tol=kw.pop("tol", 1e-3), r_min=2, r_max=kw.pop("r_max", 16),
        r_aug_max=kw.pop("r_aug_max", 32), n_mu=n_mu, n_phi=n_phi, integrator="rk4",
        inflow={"x_lo": (np.ones(ny), np.where(ox >= 0, 1.0, 0.0))},
    )
    return wl.with_(**kw) if kw else wl


def lognormal_problem(seed: int = 2602, **kw) -> Workload:
    """Scale case: [0,1]^2, 512x512 cells, 8x8 subdomains of 64x64, 2048 directions
    (32 mu x 64 phi), fixed rank 20.  sigma_t lognormal per 16x16-cell patch
    (median 1, log-sigma 1.5), scattering ratio uniform in [0.5, 1]; Gaussian
    initial data (width 0.05 at the centre); 200 steps of dt = 0.5 h."""
    nx = kw.pop("nx", 512)
    tiles = kw.pop("tiles", 8)
    patch = kw.pop("patch", 16)
    n_mu = kw.pop("n_mu", 32)
    n_phi = kw.pop("n_phi", 64)
    rank = kw.pop("rank", 20)
    nsteps = kw.pop("nsteps", 200)
    rng = np.random.default_rng(seed)
    npatch = nx // patch
    z = rng.standard_normal((npatch, npatch))
    ratio = rng.uniform(0.5, 1.0, (npatch, npatch))
    sig_t_p = np.exp(1.5 * z)
    sig_t = np.kron(sig_t_p, np.ones((patch, patch))).reshape(-1)
    rat = np.kron(ratio, np.ones((patch, patch))).reshape(-1)
    wl = gaussian_problem(name=f"lognormal-{nx}x{nx}-{tiles}x{tiles}-n{n_mu * n_phi}-r{rank}",
                          nx=nx, ny=nx, x0=0.0, x1=1.0, y0=0.0, y1=1.0, tiles_x=tiles,
                          tiles_y=tiles, n_mu=n_mu, n_phi=n_phi, centre=(0.5, 0.5),
                          width=0.05, rank=rank, nsteps=nsteps)
    wl = wl.with_(sigma_s=rat * sig_t, sigma_a=(1.0 - rat) * sig_t)
    return wl.with_(**kw) if kw else wl


def random_small_problem(seed: int, nx=8, ny=8, tiles_x=2, tiles_y=2, n_mu=2, n_phi=8,
                         rank=3, r_aug_max=6, nsteps=2, integrator="euler",
                         xcuts=None, ycuts=None) -> Workload:
    """Tiny heterogeneous problem with seeded random fields (for brute-force and
    ragged-tiling tests)."""
    rng = np.random.default_rng(seed)
    ox, oy, w = product_quadrature(n_mu, n_phi)
    nc = nx * ny
    wl = Workload(
        name=f"random-{nx}x{ny}-s{seed}", nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0,
        y1=float(ny) / nx,
        xcuts=list(xcuts) if xcuts is not None else uniform_cuts(nx, tiles_x),
        ycuts=list(ycuts) if ycuts is not None else uniform_cuts(ny, tiles_y),
        omega_x=ox, omega_y=oy, w=w,
        sigma_s=rng.uniform(0.2, 2.0, nc), sigma_a=rng.uniform(0.0, 1.0, nc),
        source=rng.uniform(0.0, 1.0, nc) * (rng.uniform(size=nc) < 0.3),
        g0=rng.uniform(0.0, 1.0, nc),
        dt=0.5 / nx, nsteps=nsteps, rank_mode="fixed", rank=rank, r_aug_max=r_aug_max,
        integrator=integrator, n_mu=n_mu, n_phi=n_phi,
    )
    return wl


def narrow_source_problem(seed: int = 13, nsteps: int = 3) -> Workload:
    """A source of width 1.5 h centred on cell (2, 2) of a 64 x 64 grid in 4 x 4
    subdomains (random heterogeneous materials, 32 directions, rank 4, RK4): the far
    subdomains start with Gaussian tails of 1e-160 .. 1e-300."""
    wl = random_small_problem(seed, nx=64, ny=64, tiles_x=4, tiles_y=4, n_mu=2, n_phi=16,
                              rank=4, r_aug_max=8, integrator="rk4", nsteps=nsteps)
    X, Y = _cell_centres(64, 64, 0.0, 1.0, 0.0, 1.0)
    h = 1.0 / 64
    g0 = np.exp(-((X - 2.5 * h) ** 2 + (Y - 2.5 * h) ** 2) / (2 * (1.5 * h) ** 2))
    return wl.with_(name="narrow-source-64x64-4x4-n32-r4", g0=g0, source=np.zeros(64 * 64))


def compact_transport_problem(tiles: int = 1, nx: int = 24, r_min: int = 4, r_max: int = 16,
                              mass_fix: bool = False, nsteps: int = 4) -> Workload:
    """Pure transport (sigma = 0, Q = 0) of a Gaussian of width 0.04 at the centre of
    [0,1]^2, far from the boundary for the first steps; 16 directions, RK4, tolerance
    mode with a tiny tolerance (1e-13) and ranks r_min..r_max."""
    wl = random_small_problem(21, nx=nx, ny=nx, tiles_x=tiles, tiles_y=tiles, n_mu=2, n_phi=8,
                              rank=2, r_aug_max=32, integrator="rk4", nsteps=nsteps)
    X, Y = _cell_centres(nx, nx, 0.0, 1.0, 0.0, 1.0)
    g0 = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.04 ** 2))
    nc = nx * nx
    return wl.with_(name=f"transport-{nx}x{nx}-{tiles}x{tiles}", sigma_s=np.zeros(nc),
                    sigma_a=np.zeros(nc), source=np.zeros(nc), g0=g0, rank_mode="tol", tol=1e-13,
                    r_min=r_min, r_max=r_max, mass_fix=mass_fix)


def random_factors(seed: int, nrow: int, n: int, r: int, hx: float, hy: float, w: np.ndarray,
                   decay: float = 0.5):
    """Seeded random low-rank factors (U, S, V) with U orthonormal in the weighted
    spatial product hx*hy*sum and V orthonormal in the quadrature product sum w.
    S has singular values decay**j.  Used only as test input."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((nrow, r))
    Qa, _ = np.linalg.qr(A)
    U = Qa / math.sqrt(hx * hy)
    B = rng.standard_normal((n, r))
    Qb, _ = np.linalg.qr(B)
    V = Qb / np.sqrt(w)[:, None]
    P, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Qr, _ = np.linalg.qr(rng.standard_normal((r, r)))
    S = P @ np.diag(decay ** np.arange(r)) @ Qr.T
    return U, S, V


DIRECTION_SETS = {128: (8, 16), 512: (16, 32), 1024: (16, 64), 16: (2, 8), 32: (4, 8)}


def batch_problems(count=64, seed0=0, grids=(64, 128, 256), tilings=(2, 4),
                   directions=(128, 512, 1024), ranks=(4, 21), nsteps=100,
                   integrator="rk4") -> dict:
    """Independent seeded problems for the batched form, grouped by direction count
    (a batch shares its direction table).  Problem i (seed seed0 + i): [0,1]^2 with a
    grid from `grids`, a square tiling from `tilings`, a direction set from
    `directions` (Gauss-Legendre mu x equidistant phi), a fixed rank drawn uniformly
    from `ranks` (inclusive; 3 r <= 64), sigma_t per 4x4 block of the grid
    log-uniform in [0.1, 100] with scattering ratio uniform in [0.5, 1], and initial
    data either a centred Gaussian of width 0.05 or a narrow Gaussian (width 1.5 h)
    at a random cell centre.  dt = h/2.  Returns {n: [Workload, ...]}."""
    out = {}
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        nx = int(rng.choice(grids))
        tiles = int(rng.choice(tilings))
        n = int(rng.choice(directions))
        n_mu, n_phi = DIRECTION_SETS[n]
        rank = int(rng.integers(ranks[0], ranks[1] + 1))
        ox, oy, w = product_quadrature(n_mu, n_phi)
        X, Y = _cell_centres(nx, nx, 0.0, 1.0, 0.0, 1.0)
        h = 1.0 / nx
        blk = nx // 4
        bs = 10.0 ** rng.uniform(-1.0, 2.0, (4, 4))
        ratio = rng.uniform(0.5, 1.0, (4, 4))
        sig_t = np.kron(bs, np.ones((blk, blk))).reshape(-1)
        rat = np.kron(ratio, np.ones((blk, blk))).reshape(-1)
        if rng.uniform() < 0.5:
            g0 = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.05 ** 2))
            kind = "gaussian"
        else:
            cx, cy = (rng.integers(0, nx, 2) + 0.5) * h
            wd = 1.5 * h
            g0 = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * wd * wd))
            kind = "point"
        wl = Workload(
            name=f"batch{i}-{nx}x{nx}-{tiles}x{tiles}-n{n}-r{rank}-{kind}", nx=nx, ny=nx,
            x0=0.0, x1=1.0, y0=0.0, y1=1.0, xcuts=uniform_cuts(nx, tiles),
            ycuts=uniform_cuts(nx, tiles), omega_x=ox, omega_y=oy, w=w,
            sigma_s=rat * sig_t, sigma_a=(1.0 - rat) * sig_t, source=np.zeros(nx * nx), g0=g0,
            dt=0.5 * h, nsteps=nsteps, rank_mode="fixed", rank=rank,
            r_aug_max=min(2 * rank, 64), integrator=integrator, n_mu=n_mu, n_phi=n_phi)
        out.setdefault(n, []).append(wl)
    return out
