"""Benchmark of the DD-DLRA time step on one GB300.

A "step" is one time step of the domain-decomposition dynamical low-rank scheme
(Algorithm 6: x-augmentation, x-advection, truncation, the same in y, then
absorption/scattering/source) on every subdomain.  The headline workload is the
largest single-GPU configuration, the lognormal medium: [0,1]^2, 512x512 cells,
8x8 subdomains of 64x64, 2048 directions (32 mu x 64 phi), fixed rank 20
(intermediate rank <= 40), lognormal sigma_t per 16x16 patch, explicit Euler,
dt = h/2, FP64.

Metric: phase-space (cell x direction) updates per second =
cells * directions * steps / time, beside the scalar-flux rel-L2 error against the
stored CPU-oracle results.  Further legs of the same JSON line: the tensor-core
forms (TF32, BF16) and the FP32-increment form on the same workload, the point
source (128^2, with its comparisons to a one-subdomain DLRA and to full-rank S_N),
the small Gaussian (against S_N), the checkerboard (full run), the 64-problem batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The default arm times the CUDA library through the C ABI; ``--impl reference``
times the CPU oracle (the plain FP64 restatement of the paper) on this machine's
host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space cell×direction updates/s; mixed vs FP64 at stated flux rel-L2 error"
UNIT = "cell-direction updates/s"
GOLD = os.path.join(ROOT, "tests", "golden")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t_local, ws, device):
    """The timed region's seconds, maximum over the ranks (each rank runs an independent
    replica of the workload; the caller brackets the region with barriers)."""
    if ws <= 1:
        return t_local
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step, steps, ws, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_step * steps * ws / seconds


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                          text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for nm, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def fp64_gemm_peak(torch):
    """Dense FP64 throughput of cuBLAS (torch.matmul, 8192^3) on this GPU, TFLOP/s."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / best / 1e12




# ---------------------------------------------------------------------------------------
# achieved rates by kernel class
# ---------------------------------------------------------------------------------------
# Slots whose kernels count their algorithmic flops (dd_dlra_profile_work: the method's
# operation count for the ranks actually used) and the roofline each is measured against;
# the m x m eigen/singular-value problems, completions and reductions are latency-bound and
# reported by time.
FP64_SLOTS = ["k_tall", "k_gram", "k_ang_coeffs", "k_sp_coeffs", "k_kstep_adv", "k_lstep_adv",
              "k_coll_kstep", "k_coll_lstep"]
TC_SLOTS = ["k_tc_tall", "k_tc_gram"]
OZ_SLOTS = ["k_oz_tall", "k_oz_gram"]   # FP64-accurate products and Grams on the BF16 tensor cores (Ozaki)
OZ_PAIRS = 28                     # digit-pair products per FP64 product (7 digits, order <= 6)
LATENCY = ["k_geig", "k_geig(aug)", "k_trunc", "k_small_adv1", "k_chol_inv", "k_sstep_adv",
           "k_coll_small", "k_kc_w", "k_kc_sel", "k_kc_apply", "k_complete", "k_reduce"]


def per_kernel_roofline(prof, nsteps, fp64_peak, fp32_peak, tc_peak, bf16_peak=None):
    """Achieved rate and fraction of each counting kernel class: the FP64 classes against
    the FP64 peak (FP32 when the form computes the class in FP32), the tensor-core classes
    against the tensor peak of their type (their three partial products counted, since the
    split is what runs); the latency classes by time."""
    out = {}
    for slot in FP64_SLOTS + TC_SLOTS + OZ_SLOTS:
        if slot not in prof or prof[slot][2] <= 0:
            continue
        ms, cnt, fl = prof[slot]
        ach = fl / (ms / 1e3) / 1e12
        if slot in OZ_SLOTS:
            out[slot] = {"ms_per_step": round(ms / nsteps, 4), "launches_per_step": cnt / nsteps,
                         "bound": "alu (integer/FP32 issue: digit conversion and recombination)",
                         "achieved_fp64_equivalent_tflops": ach,
                         "frac_of_fp64": ach / fp64_peak,
                         "achieved_bf16_tflops_28_pair_products": OZ_PAIRS * ach,
                         "frac_of_bf16_peak": OZ_PAIRS * ach / bf16_peak if bf16_peak else None}
        elif slot in TC_SLOTS:
            out[slot] = {"ms_per_step": round(ms / nsteps, 4), "launches_per_step": cnt / nsteps,
                         "bound": "tensor", "achieved_tflops_3products": 3 * ach,
                         "frac_of_tensor_peak": 3 * ach / tc_peak}
        else:
            out[slot] = {"ms_per_step": round(ms / nsteps, 4), "launches_per_step": cnt / nsteps,
                         "bound": "alu (FP64 pipe)", "achieved_tflops": ach,
                         "frac_of_fp64": ach / fp64_peak}
    out["latency_bound_ms_per_step"] = {s: round(prof[s][0] / nsteps, 4) for s in LATENCY
                                        if s in prof}
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean over one warm
# step's launches) of the kernels as they stand, from the ncu captures summarised in
# profiles/ (k_gram: profiles/k_gram_lognormal_traffic.md; k_oz_tall: the 33 launches of a
# step, profiles/k_oz_tall_lognormal.md; the lognormal workload with the tensor-core
# products).  An entry must be dropped when its kernel changes.
NCU_TRAFFIC = {"k_gram": 63.1e6, "k_oz_tall": 94.9e6}


def timed_steps(s, steps, warmup, flush, stream, torch):
    """Per-step CUDA events on the solver's stream around graph-replayed steps, L2 flushed
    (a 256 MiB write outside the events) before each; returns seconds."""
    s.step(warmup)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        s.step(1)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / 1e3


def rel(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_ours(args, torch):
    import numpy as np
    from paper_2602_14854_gb300 import binding, build
    from paper_2602_14854_gb300 import inputs

    ws, rank, local = dist_env()
    build.build()
    binding.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = inputs.lognormal_problem()
    units = wl.ncells * wl.n
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # ---- timed: the headline workload, FP64, graph-replayed steps, the launch choices
    # (tall-product engine per row family, Gram chunk counts) picked by the autotuner -------
    OPT = {"products": "auto", "autotune": True}
    s = binding.Solver(wl, stream=sptr, use_graph=True, **OPT)
    tuning, tune_ms = s.tuning()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_ours = timed_steps(s, args.steps, args.warmup, flush, stream, torch)
    if ws > 1:
        torch.distributed.barrier()
    t_ours = max_over_ranks(t_ours, ws, dev)
    value = job_value(units, args.steps, ws, t_ours)
    prof = s.profile(2, work=True)
    st_r, it_r = s.ranks()
    s.close()
    launches_per_step = sum(v[1] for v in prof.values()) / 2.0

    # ---- accuracy: the first 20 steps against the stored oracle result --------------------
    gold = np.load(os.path.join(GOLD, "lognormal_512_prefix20.npz"))
    g_steps = int(gold["nsteps"])

    def prefix_err(prec, **opt):
        sv = binding.Solver(wl, stream=sptr, use_graph=True, precision=prec, **opt)
        sv.step(g_steps)
        rho = sv.scalar_flux()
        sv.close()
        return rel(rho[gold["idx"]], gold["rho"]), rho

    err64, rho64 = prefix_err("fp64", **OPT)

    # ---- the same with the FP64 CUDA-core products throughout (no tensor cores) ------------
    sv = binding.Solver(wl, stream=sptr, use_graph=True, products="fp64")
    t_cc = timed_steps(sv, args.steps, args.warmup, flush, stream, torch)
    sv.close()
    err_cc, _ = prefix_err("fp64", products="fp64")
    cuda_core = {"ms_per_step": t_cc / args.steps * 1e3, "value": units * args.steps * ws / t_cc,
                 "unit": UNIT, "flux_rel_l2_vs_oracle_%dsteps" % g_steps: err_cc,
                 "speedup_of_headline": t_cc / t_ours}

    # ---- end to end through the public API with host buffers -------------------------------
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s3 = binding.Solver(wl, stream=sptr, use_graph=True, **OPT)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        s3.step(1)
        s3.scalar_flux()                 # device -> host read of the step's result
    t2 = time.perf_counter()
    s3.close()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_parts = {"create_ms": 1e3 * (t1 - t0), "steps_ms": 1e3 * (t2 - t1),
                 "destroy_ms": 1e3 * (time.perf_counter() - t2)}
    h2d = 8 * (4 * wl.ncells + 3 * wl.n) + 4 * (len(wl.xcuts) + len(wl.ycuts))
    e2e = {"value": units * args.steps * ws / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 8 * wl.ncells,
           "note": "create (problem data from host memory; the autotuner's choices cached "
                   "from the first solver of this shape) + per step: step + scalar flux to "
                   "host + destroy, wall clock", "parts": e2e_parts}

    # ---- roofline ------------------------------------------------------------------------
    peaks = measured_peaks()
    fp64_peak = fp64_gemm_peak(torch)
    bf16_peak = peaks.get("bf16_tflops") or 1900.0
    kernels = per_kernel_roofline(prof, 2, fp64_peak, None, bf16_peak / 2.0, bf16_peak)
    total = sum(v[0] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][0])
    roof = {"kernel": top[0], "bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak,
            "peak_source": "cuBLAS FP64 GEMM 8192^3 measured in this run (of measured)",
            "share_of_step": top[1][0] / total, "launch_ms": top[1][0] / top[1][1],
            "launches_per_step": top[1][1] / 2.0, "traffic": NCU_TRAFFIC.get(top[0])}
    if top[0] in OZ_SLOTS and top[1][2] > 0:
        ach = top[1][2] / (top[1][0] / 1e3) / 1e12
        roof.update({"achieved": ach, "frac": ach / fp64_peak,
                     "note": "FP64-accurate products on the BF16 tensor cores: achieved is the "
                             "FP64 work per second, against the FP64 roofline",
                     "work_flops_per_launch": top[1][2] / top[1][1],
                     "work_source": "counted by the kernels (dd_dlra_profile_work)"})
    elif top[1][2] > 0:
        ach = top[1][2] / (top[1][0] / 1e3) / 1e12
        roof.update({"achieved": ach, "frac": ach / fp64_peak,
                     "work_flops_per_launch": top[1][2] / top[1][1],
                     "work_source": "counted by the kernels (dd_dlra_profile_work)"})
    else:
        roof.update({"achieved": None, "frac": None, "note": "latency-bound: time only"})
    roof["kernels"] = kernels
    roof["kernels_ms_per_step"] = {k: round(v[0] / 2.0, 4) for k, v in
                                   sorted(prof.items(), key=lambda kv: -kv[1][0])}

    # ---- the reduced-precision forms on the same workload ---------------------------------
    forms = {}
    if not args.no_mixed:
        for prec in ("tf32", "bf16", "mixed"):
            sv = binding.Solver(wl, stream=sptr, use_graph=True, precision=prec, **OPT)
            t_p = timed_steps(sv, args.steps, args.warmup, flush, stream, torch)
            pp = sv.profile(1, work=True)
            sv.close()
            e_or, rho_p = prefix_err(prec, **OPT)
            forms[prec] = {"value": units * args.steps * ws / t_p, "unit": UNIT,
                           "ms_per_step": t_p / args.steps * 1e3, "speedup_vs_fp64": t_ours / t_p,
                           "flux_rel_l2_vs_oracle_%dsteps" % g_steps: e_or,
                           "flux_rel_l2_vs_fp64_%dsteps" % g_steps: rel(rho_p, rho64),
                           "kernels_ms_per_step": {k: round(v[0], 4) for k, v in
                                                   sorted(pp.items(), key=lambda kv: -kv[1][0])[:8]},
                           "kernels": per_kernel_roofline(pp, 1, fp64_peak, None,
                                                          bf16_peak / (2.0 if prec == "tf32" else 1.0),
                                                          bf16_peak)}
        forms["note"] = ("tf32/bf16: Galerkin contractions as tcgen05 MMAs (operands split "
                         "hi + lo, FP32 accumulation), FP32 increments; mixed: FP32 "
                         "increments only; orthonormalisations, QR R factors, SVDs, eigen-"
                         "splits and the K-step FP64-accurate in every form (the tall "
                         "products of the orthonormalisations on the Ozaki kernel where the "
                         "autotuner picks it)")

    # ---- the point source: oracle, one-subdomain DLRA, full-rank S_N ---------------------
    point = None
    if not args.no_legs:
        wp = inputs.config_c1()
        g1 = np.load(os.path.join(GOLD, "pointsource_128_rk4_t1.npz"))
        sn_ref = np.load(os.path.join(GOLD, "sn_reference.npz"))
        sv = binding.Solver(wp, stream=sptr, use_graph=True)
        t_p = timed_steps(sv, args.steps, args.warmup, flush, stream, torch)
        sv.close()
        runs = {}
        for prec in ("fp64", "tf32", "bf16"):
            sv = binding.Solver(wp, stream=sptr, use_graph=True, precision=prec)
            sv.step(wp.nsteps)
            runs[prec] = sv.scalar_flux()
            sv.close()
        w11 = wp.with_(xcuts=[0, wp.nx], ycuts=[0, wp.ny])     # classic DLRA, rank 10
        sv = binding.Solver(w11, stream=sptr, use_graph=True)
        sv.step(w11.nsteps)
        rho11 = sv.scalar_flux()
        sv.close()
        point = {"workload": wp.name, "value": wp.ncells * wp.n * args.steps * ws / t_p,
                 "unit": UNIT, "ms_per_step": t_p / args.steps * 1e3,
                 "flux_rel_l2_vs_oracle": {p: rel(r, g1["rho"]) for p, r in runs.items()},
                 "flux_rel_l2_vs_one_subdomain_dlra_r10": rel(runs["fp64"], rho11),
                 "flux_rel_l2_vs_full_rank_sn": rel(runs["fp64"], sn_ref["pointsource"]),
                 "one_subdomain_dlra_r10_vs_full_rank_sn": rel(rho11, sn_ref["pointsource"]),
                 "steps": wp.nsteps}
        w0 = inputs.config_c0()
        sv = binding.Solver(w0, stream=sptr, use_graph=True)
        sv.step(w0.nsteps)
        point["gaussian32_flux_rel_l2_vs_full_rank_sn"] = rel(sv.scalar_flux(), sn_ref["gaussian32"])
        sv.close()

    # ---- the checkerboard: full run against the stored oracle result ----------------------
    checker = None
    if not args.no_legs:
        wc = inputs.checkerboard_problem()
        gc = np.load(os.path.join(GOLD, "checkerboard_224_full.npz"))
        sv = binding.Solver(wc, stream=sptr, use_graph=True)
        t_c = timed_steps(sv, args.steps, args.warmup, flush, stream, torch)
        sv.close()
        sv = binding.Solver(wc, stream=sptr, use_graph=True)
        sv.step(wc.nsteps)
        rc_ = sv.scalar_flux()
        sv.close()
        checker = {"workload": wc.name, "value": wc.ncells * wc.n * args.steps * ws / t_c,
                   "unit": UNIT, "ms_per_step": t_c / args.steps * 1e3, "steps": wc.nsteps,
                   "flux_rel_l2_vs_oracle_full_run": rel(rc_, gc["rho"])}
        sp_path = os.path.join(GOLD, "checkerboard_224_spread.npz")
        if os.path.exists(sp_path):
            checker["oracle_spread_under_1e-13_direction_noise"] = rel(np.load(sp_path)["rho"],
                                                                       gc["rho"])

    # ---- batched form ----------------------------------------------------------------
    batch = None
    if args.batch > 0:
        batch = run_batch(args, torch, dev, flush)

    # ---- CPU baseline: the oracle on this machine's host cores ------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(nsteps=args.cpu_steps)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ours / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "cells": wl.ncells, "directions": wl.n,
                   "subdomains": wl.nsub, "rank": wl.rank, "r_aug_max": wl.r_aug_max,
                   "integrator": wl.integrator, "dt": wl.dt, "parallelism": f"replicas{ws}",
                   "l2": "flushed between timed steps (256 MiB write, outside the step events); "
                         "the factors alone (~250 MB) exceed L2",
                   "launch": "one CUDA graph per step",
                   "options": "products=auto, autotune=1 (the choices in 'tuning')"},
        "tuning": {"choices": tuning, "trial_ms": tune_ms},
        "fp64_cuda_core_products": cuda_core,
        "flux_rel_l2_vs_oracle_%dsteps" % g_steps: err64,
        "ranks": {"stored_max": int(np.max(st_r)), "intermediate_max": int(np.max(it_r))},
        "e2e": e2e,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "gpu_launches_per_step": launches_per_step,
        "roofline": roof,
        "clocks": clk.summary(),
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                  "fp64_gemm_tflops": fp64_peak},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if forms:
        line["forms"] = forms
    if point is not None:
        line["pointsource"] = point
    if checker is not None:
        line["checkerboard"] = checker
    if batch is not None:
        line["batch"] = batch
    return line, rank


def run_batch(args, torch, dev, flush):
    """The batched form: 64 seeded independent problems (grids 64^2/128^2/256^2, 2x2 or
    4x4 tilings, 128/512/1024 directions, ranks 4..21, RK4), one solver per direction
    count, the three solvers replayed concurrently on three streams.  Timed in FP64, in the
    tensor-core forms and in the FP32-increment form, beside the plain FP64 loop (one solver
    per problem, one after another).  Each form's flux is compared with the FP64 flux of the
    same run, beside each problem's FP64 sensitivity to 1e-7 noise on its initial data and on
    its direction components."""
    import numpy as np
    from paper_2602_14854_gb300 import binding, inputs
    groups = sorted(inputs.batch_problems(count=args.batch).items())
    units = sum(w.ncells * w.n for _, wls in groups for w in wls)
    K = args.batch_steps
    main = torch.cuda.current_stream(dev)

    def timed(solvers, streams):
        for sv in solvers:
            sv.step(args.warmup)
        torch.cuda.synchronize()
        flush.fill_(1.0)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(main)
        ends = []
        for sv, st in zip(solvers, streams):
            st.wait_event(t0)
            sv.step(K)
            e = torch.cuda.Event()
            e.record(st)
            ends.append(e)
        for e in ends:
            main.wait_event(e)
        t1.record(main)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3

    out = {"workload": f"batch{args.batch}: 64^2/128^2/256^2 grids, 2x2/4x4 tilings, "
                       "128/512/1024 directions, ranks 4-21, RK4",
           "problems": args.batch, "steps": K, "warmup": args.warmup,
           "groups": [{"directions": n, "problems": len(wls),
                       "cells": sum(w.ncells for w in wls)} for n, wls in groups],
           "l2": "working set (tall factors of all problems) larger than L2"}
    flux = {}
    for prec in ("fp64", "tf32", "bf16", "mixed"):
        streams = [torch.cuda.Stream(dev) for _ in groups]
        solvers = [binding.Solver(wls, stream=st.cuda_stream, use_graph=True, precision=prec)
                   for (n, wls), st in zip(groups, streams)]
        t = timed(solvers, streams)
        flux[prec] = [sv.scalar_flux() for sv in solvers]
        launches = 0
        if prec == "fp64":
            launches = sum(c for sv in solvers for _, c in sv.profile(1).values())
        for sv in solvers:
            sv.close()
        out[prec] = {"value": units * K / t, "unit": UNIT, "ms_per_step": t / K * 1e3}
        if launches:
            out[prec]["gpu_launches_per_step"] = launches

    def fp64_flux(perturb, seed):
        rng = np.random.default_rng(seed)
        out_ = []
        for n, wls in groups:
            sv = binding.Solver(perturb(wls, rng), stream=main.cuda_stream, use_graph=True)
            sv.step(args.warmup + K)
            out_.append(sv.scalar_flux())
            sv.close()
        return out_

    def noise(rng, shape):
        return 1.0 + 1e-7 * rng.uniform(-1.0, 1.0, shape)

    def p_g0(wls, rng):
        return [w.with_(g0=w.g0 * noise(rng, w.g0.shape)) for w in wls]

    def p_dir(wls, rng):      # one direction table per group: the same noise for all
        a, b = noise(rng, wls[0].omega_x.shape), noise(rng, wls[0].omega_y.shape)
        return [w.with_(omega_x=w.omega_x * a, omega_y=w.omega_y * b) for w in wls]

    pert = {"initial_data": fp64_flux(p_g0, 7), "directions": fp64_flux(p_dir, 11)}
    errs = {p: [] for p in ("tf32", "bf16", "mixed")}
    spread = {kk: [] for kk in pert}
    for gi, (n, wls) in enumerate(groups):
        lo = 0
        for w in wls:
            sl = slice(lo, lo + w.ncells)
            lo += w.ncells
            ref = flux["fp64"][gi][sl]
            nr = max(np.linalg.norm(ref), 1e-300)
            for p in errs:
                errs[p].append(float(np.linalg.norm(flux[p][gi][sl] - ref) / nr))
            for kk, pv in pert.items():
                spread[kk].append(float(np.linalg.norm(pv[gi][sl] - ref) / nr))
    spread = {kk: np.array(v) for kk, v in spread.items()}
    worst = np.maximum.reduce(list(spread.values()))
    out["fp64_sensitivity_to_1e-7_noise"] = {
        kk: {"max": float(v.max()), "median": float(np.median(v)),
             "problems_above_1e-6": int(np.sum(v > 1e-6))} for kk, v in spread.items()}
    for p, bound in (("tf32", 1e-5), ("bf16", 1e-3), ("mixed", 1e-5)):
        e = np.array(errs[p])
        out[p].update({
            "flux_rel_l2_vs_fp64_max": float(e.max()),
            "flux_rel_l2_vs_fp64_median": float(np.median(e)),
            f"problems_within_{bound:g}": int(np.sum(e <= bound)),
            # a problem whose FP64 result moves by more than a tenth of the bound under 1e-7
            # noise on its data is too ill-conditioned for FP32-level arithmetic to hold it
            f"problems_within_{bound:g}_or_ill_conditioned": int(np.sum((e <= bound) | (worst > 0.1 * bound))),
            "max_error_on_well_conditioned": float(np.max(e[worst <= 0.1 * bound]))
            if np.any(worst <= 0.1 * bound) else None,
            "speedup_vs_fp64_batched": out["fp64"]["ms_per_step"] / out[p]["ms_per_step"]})

    # plain FP64 loop: one solver per problem, replayed one after another
    singles = [binding.Solver(w, stream=main.cuda_stream, use_graph=True)
               for _, wls in groups for w in wls]
    for sv in singles:
        sv.step(args.warmup)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(main)
    for _ in range(K):
        for sv in singles:
            sv.step(1)
    t1.record(main)
    torch.cuda.synchronize()
    t = t0.elapsed_time(t1) / 1e3
    for sv in singles:
        sv.close()
    out["fp64_loop"] = {"value": units * K / t, "unit": UNIT, "ms_per_step": t / K * 1e3}
    for p in ("fp64", "tf32", "bf16", "mixed"):
        out[p]["speedup_vs_fp64_loop"] = out["fp64_loop"]["ms_per_step"] / out[p]["ms_per_step"]
    return out


def sample_workload():
    """The bounded sample of the headline workload the CPU oracle is timed on: the same
    subdomains (64x64 cells, 2048 directions, rank 20, r_t <= 40, lognormal medium), 2x2 of
    them (128^2 cells) instead of 8x8."""
    from paper_2602_14854_gb300 import inputs
    return inputs.lognormal_problem(nx=128, tiles=2)


def cpu_baseline(nsteps=2):
    from oracle import dd_dlra
    wl = sample_workload()
    o = dd_dlra.DDDLRA(wl)
    o.step()                                # first step excluded (start-up)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        o.step()
    t = time.perf_counter() - t0
    return {"value": wl.ncells * wl.n * nsteps / t, "unit": UNIT,
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{nsteps} time steps (steps 2..{nsteps + 1}) of {wl.name}: the headline "
                      f"workload's subdomains, 2x2 of them instead of 8x8; numpy FP64 with "
                      f"multithreaded BLAS, {t:.1f} s"}


def run_reference(args):
    """The CPU oracle timed as the reference arm (rank 0 only), on the bounded sample of
    the headline workload."""
    from oracle import dd_dlra
    ws, rank, _ = dist_env()
    if rank != 0:
        return None, rank
    wl = sample_workload()
    o = dd_dlra.DDDLRA(wl)
    for _ in range(args.warmup):
        o.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step()
    t = time.perf_counter() - t0
    value = wl.ncells * wl.n * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "lognormal-512x512-8x8-n2048-r20 (bounded sample: " + wl.name + ")",
                       "cells": wl.ncells, "directions": wl.n, "subdomains": wl.nsub,
                       "rank": wl.rank, "integrator": wl.integrator},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{args.steps} full time steps after {args.warmup} warm-up "
                                       f"steps of {wl.name}, the headline workload's subdomains "
                                       "(2x2 of them instead of 8x8)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    return line, rank


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-legs", action="store_true")
    ap.add_argument("--batch", type=int, default=64,
                    help="problems of the batched leg (0 skips it)")
    ap.add_argument("--batch-steps", type=int, default=10)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if ws > 1 and rank != 0:
            return
        line, rank = run_reference(args)
        if line is not None:
            print(json.dumps(line))
        return
    import torch
    if ws > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    line, rank = run_ours(args, torch)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
