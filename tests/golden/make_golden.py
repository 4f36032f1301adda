"""Write the stored expected values of the GPU parity tests and of the benchmark's
accuracy figures.

Calls only the CPU oracle (oracle/) on the seeded synthetic workloads of
paper_2602_14854_gb300.inputs.  Run from the repository root, naming the targets:

    python tests/golden/make_golden.py pointsource checkerboard lognormal20 \
        batch10 batch100 sn

pointsource   point source (128^2, 4x4, 512 directions, rank 10, RK4), 86 steps to t = 1:
              the whole scalar flux and the stored ranks.
checkerboard  checkerboard (224^2, 7x7, 1024 directions, tolerance 1e-4), all 205 steps:
              the whole scalar flux, the stored ranks after every step.
lognormal20   lognormal medium (512^2, 8x8, 2048 directions, rank 20), the first 20 of its
              200 steps (the oracle needs about a minute per step on 8 host cores): the
              scalar flux on 16384 seeded cells, the norm of the whole flux, the ranks.
batch10       the 64 batch problems (batch_problems()), each over the first 10 of its 100
              steps: the scalar flux on up to 2048 seeded cells, its whole norm, the ranks.
batch100      the batch problems listed in BATCH_FULL over all 100 steps (the oracle needs
              about 14 CPU-hours for all 64 over 100 steps; these are a seeded sample of
              one in eight, with every direction count and tiling represented).
sn            the full-rank S_N solution (oracle/sn.py) of the small Gaussian (50 Euler
              steps) and of the point source (86 RK4 steps): the scalar flux.
batch1        the 64 batch problems over one step (per-step parity before any amplification).
batch10_stepnoise, batch100_stepnoise
              the sensitive batch problems (SENSITIVE_*) with the core S of every subdomain
              perturbed by a seeded relative 1e-13 after every step.
checkerboard_spread, batch10_spread, batch100_spread
              the same oracle runs from direction components perturbed by a seeded relative
              1e-13 (rounding-sized, symmetry-breaking noise): how far the problem's own
              result moves under perturbations of the size rounding makes, stored beside
              the unperturbed result (the tests bound the GPU's difference by it where it
              exceeds 1e-9).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dd_dlra, sn  # noqa: E402
from paper_2602_14854_gb300 import inputs  # noqa: E402

BATCH_FULL = (0, 3, 9, 17, 30, 35, 48, 58)
# the batch problems whose FP64 GPU result differs from the stored oracle result by more than
# 1e-9 (narrow point sources; their stored values are the oracle's, like every other)
SENSITIVE_PREFIX = (20, 22, 29, 32, 33, 43)
SENSITIVE_FULL = (0, 9, 35, 48, 58)


def sample_cells(ncells, count, seed):
    """Seeded sorted sample of cell indices (all cells when count >= ncells)."""
    if count >= ncells:
        return np.arange(ncells)
    return np.sort(np.random.default_rng(seed).choice(ncells, count, replace=False))


def pointsource():
    wl = inputs.config_c1()
    t = time.time()
    o = dd_dlra.DDDLRA(wl)
    o.run()
    rho = o.scalar_flux()
    np.savez_compressed(os.path.join(HERE, "pointsource_128_rk4_t1.npz"), rho=rho,
                        ranks=np.array(o.ranks()), nsteps=wl.nsteps, dt=wl.dt)
    print(f"point source: {wl.nsteps} steps in {time.time() - t:.1f} s, ranks {o.ranks()}")


def checkerboard():
    wl = inputs.checkerboard_problem()
    t = time.time()
    o = dd_dlra.DDDLRA(wl)
    hist = []
    for _ in range(wl.nsteps):
        o.step()
        hist.append(o.ranks())
    np.savez_compressed(os.path.join(HERE, "checkerboard_224_full.npz"), rho=o.scalar_flux(),
                        ranks=np.array(hist, dtype=np.int16), nsteps=wl.nsteps)
    print(f"checkerboard: {wl.nsteps} steps in {time.time() - t:.1f} s, ranks {o.ranks()}")


def lognormal20(nsteps=20):
    wl = inputs.lognormal_problem()
    t = time.time()
    o = dd_dlra.DDDLRA(wl)
    o.run(nsteps)
    rho = o.scalar_flux()
    idx = sample_cells(wl.ncells, 16384, 2602)
    np.savez_compressed(os.path.join(HERE, "lognormal_512_prefix20.npz"), idx=idx, rho=rho[idx],
                        norm=np.linalg.norm(rho), ranks=np.array(o.ranks()), nsteps=nsteps)
    print(f"lognormal: {nsteps} steps in {time.time() - t:.1f} s, ranks {o.ranks()}")


def batch(nsteps, which, fname):
    out = {}
    t = time.time()
    probs = {int(w.name.split("-")[0][5:]): w
             for wls in inputs.batch_problems(count=64).values() for w in wls}
    for i in which:
        wl = probs[i]
        o = dd_dlra.DDDLRA(wl)
        o.run(nsteps)
        rho = o.scalar_flux()
        idx = sample_cells(wl.ncells, 2048, 1000 + i)
        out[f"p{i}_idx"] = idx
        out[f"p{i}_rho"] = rho[idx]
        out[f"p{i}_norm"] = np.linalg.norm(rho)
        out[f"p{i}_ranks"] = np.array(o.ranks())
        print(f"  {wl.name}: {time.time() - t:.0f} s", flush=True)
        np.savez_compressed(os.path.join(HERE, fname), nsteps=nsteps,
                            problems=np.array(sorted(int(k[1:].split("_")[0]) for k in out
                                                     if k.endswith("_norm"))), **out)
    print(f"batch ({nsteps} steps, {len(which)} problems): {time.time() - t:.1f} s")


def perturbed(wl, seed):
    """The workload with its direction components scaled by 1 + 1e-13 u, u ~ U[-1, 1]."""
    rng = np.random.default_rng(seed)
    return wl.with_(omega_x=wl.omega_x * (1.0 + 1e-13 * rng.uniform(-1.0, 1.0, wl.n)),
                    omega_y=wl.omega_y * (1.0 + 1e-13 * rng.uniform(-1.0, 1.0, wl.n)))


def checkerboard_spread():
    wl = perturbed(inputs.checkerboard_problem(), 77)
    t = time.time()
    o = dd_dlra.DDDLRA(wl)
    hist = []
    for _ in range(wl.nsteps):
        o.step()
        hist.append(o.ranks())
    np.savez_compressed(os.path.join(HERE, "checkerboard_224_spread.npz"), rho=o.scalar_flux(),
                        ranks=np.array(hist, dtype=np.int16), nsteps=wl.nsteps)
    print(f"checkerboard (perturbed): {time.time() - t:.1f} s", flush=True)


def batch_spread(nsteps, which, fname):
    out = {}
    t = time.time()
    probs = {int(w.name.split("-")[0][5:]): w
             for wls in inputs.batch_problems(count=64).values() for w in wls}
    for i in which:
        wl = perturbed(probs[i], 500 + i)
        o = dd_dlra.DDDLRA(wl)
        o.run(nsteps)
        rho = o.scalar_flux()
        idx = sample_cells(wl.ncells, 2048, 1000 + i)
        out[f"p{i}_rho"] = rho[idx]
        out[f"p{i}_ranks"] = np.array(o.ranks())
        print(f"  {wl.name} (perturbed): {time.time() - t:.0f} s", flush=True)
        np.savez_compressed(os.path.join(HERE, fname), nsteps=nsteps,
                            problems=np.array(sorted(int(k[1:].split("_")[0]) for k in out
                                                     if k.endswith("_rho"))), **out)


def batch_stepnoise(nsteps, which, fname, rel=1e-13):
    """The oracle with every subdomain's core S multiplied by (1 + rel u), u ~ U[-1, 1]
    seeded, after every step: how far differences of the size one FP64 step leaves
    between two correct implementations (measured: ~1e-13 relative after one step) move the
    result over nsteps steps."""
    out = {}
    t = time.time()
    probs = {int(w.name.split("-")[0][5:]): w
             for wls in inputs.batch_problems(count=64).values() for w in wls}
    for i in which:
        wl = probs[i]
        rng = np.random.default_rng(700 + i)
        o = dd_dlra.DDDLRA(wl)
        for _ in range(nsteps):
            o.step()
            o.state = [(U, S * (1.0 + rel * rng.uniform(-1.0, 1.0, S.shape)), V)
                       for U, S, V in o.state]
        rho = o.scalar_flux()
        idx = sample_cells(wl.ncells, 2048, 1000 + i)
        out[f"p{i}_rho"] = rho[idx]
        out[f"p{i}_ranks"] = np.array(o.ranks())
        print(f"  {wl.name} (noise after every step): {time.time() - t:.0f} s", flush=True)
        np.savez_compressed(os.path.join(HERE, fname), nsteps=nsteps, rel=rel,
                            problems=np.array(sorted(int(k[1:].split("_")[0]) for k in out
                                                     if k.endswith("_rho"))), **out)


def sn_refs():
    out = {}
    for key, wl in (("gaussian32", inputs.config_c0()), ("pointsource", inputs.config_c1())):
        t = time.time()
        out[key] = sn.scalar_flux(sn.run(wl), wl)
        print(f"S_N {key}: {wl.nsteps} steps in {time.time() - t:.1f} s")
    np.savez_compressed(os.path.join(HERE, "sn_reference.npz"), **out)


TARGETS = {
    "pointsource": pointsource,
    "checkerboard": checkerboard,
    "lognormal20": lognormal20,
    "batch10": lambda: batch(10, range(64), "batch64_prefix10.npz"),
    "batch100": lambda: batch(100, BATCH_FULL, "batch64_sample_full.npz"),
    "sn": sn_refs,
    "checkerboard_spread": checkerboard_spread,
    "batch10_spread": lambda: batch_spread(10, range(64), "batch64_prefix10_spread.npz"),
    "batch100_spread": lambda: batch_spread(100, BATCH_FULL, "batch64_sample_full_spread.npz"),
    "batch1": lambda: batch(1, range(64), "batch64_step1.npz"),
    "batch10_stepnoise": lambda: batch_stepnoise(10, SENSITIVE_PREFIX, "batch64_prefix10_stepnoise.npz"),
    "batch100_stepnoise": lambda: batch_stepnoise(100, SENSITIVE_FULL, "batch64_sample_full_stepnoise.npz"),
}


if __name__ == "__main__":
    for name in sys.argv[1:] or ["pointsource"]:
        TARGETS[name]()
