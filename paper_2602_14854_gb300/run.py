"""Run the DD-DLRA time step on one of the synthetic workloads and print a JSON
summary (scalar-flux statistics, ranks, wall time).

    python -m paper_2602_14854_gb300.run --workload pointsource --steps 20 [--graph]
        [--precision fp64|mixed|tf32|bf16] [--products fp64|tensor|auto] [--autotune]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from paper_2602_14854_gb300 import binding, build, inputs

WORKLOADS = {
    "gaussian32": lambda: inputs.config_c0(),
    "gaussian32-rk4": lambda: inputs.config_c0(integrator="rk4"),
    "pointsource": lambda: inputs.config_c1(),
    "checkerboard": lambda: inputs.checkerboard_problem(),
    "lognormal": lambda: inputs.lognormal_problem(),
    "hohlraum": lambda: inputs.hohlraum_problem(),
}


def run_batch(args):
    """The 64-problem batch, one solver per direction count."""
    groups = inputs.batch_problems(count=args.batch, nsteps=args.steps or 100)
    out = {"workload": f"batch{args.batch}", "groups": []}
    total_units, total_t = 0.0, 0.0
    for n, wls in sorted(groups.items()):
        s = binding.Solver(wls, use_graph=args.graph, precision=args.precision,
                           products=args.products, autotune=args.autotune)
        s.step(args.warmup)
        s.sync()
        nsteps = args.steps or 100
        t0 = time.perf_counter()
        s.step(nsteps)
        s.sync()
        t = time.perf_counter() - t0
        units = sum(w.ncells for w in wls) * n * nsteps
        total_units += units
        total_t += t
        g = {"directions": n, "problems": len(wls), "subdomains": s.nsub, "seconds": t,
             "updates_per_s": units / t}
        if args.profile:
            prof = s.profile(args.profile)
            g["profile_ms"] = {k: [round(v[0], 3), v[1]] for k, v in
                               sorted(prof.items(), key=lambda kv: -kv[1][0])[:8]}
        out["groups"].append(g)
        s.close()
    out["updates_per_s"] = total_units / total_t
    print(json.dumps(out))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="pointsource", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--profile", type=int, default=0,
                    help="additionally advance this many steps with per-kernel event timing")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "tf32", "bf16"])
    ap.add_argument("--products", default="fp64", choices=["fp64", "tensor", "auto"],
                    help="engine of the FP64 tall products (dd_options.products)")
    ap.add_argument("--autotune", action="store_true",
                    help="time the launch choices when the solver is created")
    ap.add_argument("--batch", type=int, default=0,
                    help="run the batched form on this many seeded problems instead")
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args(argv)
    build.build()
    if args.batch:
        run_batch(args)
        return
    wl = WORKLOADS[args.workload]()
    nsteps = wl.nsteps if args.steps is None else args.steps
    s = binding.Solver(wl, use_graph=args.graph, precision=args.precision,
                       products=args.products, autotune=args.autotune)
    t0 = time.perf_counter()
    s.step(nsteps)
    s.sync()
    t = time.perf_counter() - t0
    prof = s.profile(args.profile) if args.profile else None
    rho = s.scalar_flux()
    stored, inter = s.ranks()
    out = {"workload": wl.name, "steps": nsteps, "seconds": t,
           "updates_per_s": wl.ncells * wl.n * nsteps / t,
           "rho_sum": float(np.sum(rho)), "rho_max": float(np.max(rho)),
           "ranks": stored.tolist(), "intermediate": inter.tolist(),
           "tuning": s.tuning()[0]}
    if prof:
        out["profile_ms"] = {k: [round(v[0], 4), v[1]] for k, v in
                             sorted(prof.items(), key=lambda kv: -kv[1][0])}
    s.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
