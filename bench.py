"""Benchmark of the DD-DLRA time step on one GB300.

A "step" is one time step of the domain-decomposition dynamical low-rank
scheme (Algorithm 6: x-augmentation, x-advection, truncation, the same in y,
then absorption/scattering/source) on every subdomain of the point-source
workload: [-1.5,1.5]^2, 128x128 cells, 4x4 subdomains of 32x32, 512 directions
(16 mu x 32 phi), rank 10 (intermediate rank <= 20), RK4, dt = 1/86.

Metric: phase-space (cell x direction) updates per second =
cells * directions * steps / time, FP64, with the scalar-flux rel-L2 error of
a full run (86 steps to t = 1) against the stored CPU-oracle result.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The default arm times the CUDA library through the C ABI; ``--impl reference``
times the CPU oracle (the plain FP64 restatement of the paper) on this
machine's host cores.
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
GOLDEN = os.path.join(ROOT, "tests", "golden", "pointsource_128_rk4_t1.npz")


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


def kernel_work(name, wl, rt, rs):
    """Algorithmic FP64 flops of one launch of a kernel class on this workload
    (rt: intermediate rank, rs: stored rank; uniform subdomains).  The symmetric
    eigendecompositions count 9 m^3 per m x m problem (the textbook cost of a
    tridiagonal-QR eigensolver with vectors), whatever the method that runs."""
    nsub = wl.nsub
    N = wl.ncells // nsub
    n = wl.n
    st = 4 if wl.integrator == "rk4" else 1
    if name == "k_kstep_adv":      # FP64 eigen-split: K P and the increment times P^T
        # (2 r_t^2 flops each per cell) plus ~10 flops per entry per stage in the eigenbasis
        return nsub * N * (4 * rt * rt + 10 * rt * st)
    if name == "k_lstep_adv":      # (r_t x r_t) matvec per direction per stage + S2 v
        return nsub * n * (2 * rt * rt * st + 4 * rt * rt)
    if name == "k_geig":           # 4 advection QRs (m = r_t) and 2 collision QRs (m = r)
        return nsub * 9 * (4 * rt ** 3 + 2 * rs ** 3) / 6.0
    if name == "k_geig(aug)":      # augmentation input of 3 r columns
        return nsub * 9 * (3 * rs) ** 3
    return None


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu
# captures summarised in profiles/k_geig_k_gram_k_tall_k_kc_pointsource_full.md and
# profiles/k_kstep_eig_k_lstep_adv_pointsource_full.md (k_kstep_adv is the profile name of
# the FP64 K-step, the eigenbasis kernel k_kstep_eig); one captured launch each (k_geig: a
# QR with m = 20 over 8 chunk partials; k_gram: the 16-chunk launch over the spatial K;
# k_tall: the 512-CTA launch over the spatial rows, from profiles/k_tall_pointsource_full.md).
# None where no capture of the kernel as it stands exists.
NCU_TRAFFIC = {"k_geig": 0.419e6, "k_kstep_adv": 3.57e6, "k_gram": 2.40e6, "k_tall": 3.21e6}


def run_ours(args, torch):
    from paper_2602_14854_gb300 import binding, build
    from paper_2602_14854_gb300 import inputs

    ws, rank, local = dist_env()
    build.build()
    binding.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = inputs.config_c1()
    units = wl.ncells * wl.n
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    # ---- timed: graph-replayed steps, L2 flushed between steps -------------------------
    s = binding.Solver(wl, stream=sptr, use_graph=True)
    s.step(args.warmup)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            s.step(1)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ours = max_over_ranks(sum(step_ms) / 1e3, ws, dev)
    value = job_value(units, args.steps, ws, t_ours)

    # ---- per-kernel profile (event pair around every launch), 4 steps ------------------
    prof = s.profile(4)
    st_r, it_r = s.ranks()
    s.close()
    total = sum(v[0] for v in prof.values())
    launches_per_step = sum(v[1] for v in prof.values()) / 4.0
    top = max(prof.items(), key=lambda kv: kv[1][0])

    # ---- accuracy of a full run against the stored oracle result ----------------------
    err = None
    if os.path.exists(GOLDEN):
        g = np.load(GOLDEN)
        s2 = binding.Solver(wl, stream=sptr, use_graph=True)
        s2.step(wl.nsteps)
        rho = s2.scalar_flux()
        s2.close()
        err = float(np.linalg.norm(rho - g["rho"]) / np.linalg.norm(g["rho"]))

    # ---- end to end through the public API with host buffers ---------------------------
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s3 = binding.Solver(wl, stream=sptr, use_graph=True)
    out = None
    for _ in range(args.steps):
        s3.step(1)
        out = s3.scalar_flux()          # device -> host read of the step's result
    s3.close()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    h2d = 8 * (3 * wl.ncells + wl.ncells + 3 * wl.n) + 4 * (len(wl.xcuts) + len(wl.ycuts))
    e2e = {"value": units * args.steps * ws / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 8 * wl.ncells,
           "note": "create (problem data upload) + per step: step + scalar flux to host + destroy"}
    del out

    # ---- roofline of the dominant kernel -----------------------------------------------
    peaks = measured_peaks()
    fp64_peak = fp64_gemm_peak(torch)
    rt = int(np.max(it_r)) if it_r.size else wl.r_aug_max
    rs = int(np.max(st_r)) if st_r.size else wl.rank
    name, (ms, cnt) = top
    work = kernel_work(name, wl, rt, rs)
    roof = {"kernel": name, "bound": "alu", "unit": "TFLOP/s", "peak": fp64_peak,
            "peak_source": "cuBLAS FP64 GEMM 8192^3 measured in this run (of measured)",
            "share_of_step": ms / total, "launch_ms": ms / cnt,
            "traffic": NCU_TRAFFIC.get(name)}
    if work is not None:
        ach = work / (ms / cnt / 1e3) / 1e12
        roof.update({"achieved": ach, "frac": ach / fp64_peak, "work_flops_per_launch": work})
    else:
        roof.update({"achieved": None, "frac": None})
    if name.startswith("k_geig"):
        roof["note"] = ("one CTA per subdomain (16 of 152 SMs) running Jacobi sweeps: latency-"
                        "bound (ncu: 14% issue-active, 15% FP64 pipe on its SMs, 0.09% of DRAM "
                        "bandwidth; Jacobi sweeps 56%, pivoted Cholesky 23% of its cycles)")
    kstep = prof.get("k_kstep_adv")
    if kstep:
        w = kernel_work("k_kstep_adv", wl, rt, rs)
        roof["k_kstep_adv"] = {"launch_ms": kstep[0] / kstep[1],
                               "achieved_tflops": w / (kstep[0] / kstep[1] / 1e3) / 1e12,
                               "frac": w / (kstep[0] / kstep[1] / 1e3) / 1e12 / fp64_peak,
                               "traffic": NCU_TRAFFIC.get("k_kstep_adv")}
    roof["kernels_ms_per_step"] = {k: round(v[0] / 4.0, 4) for k, v in
                                   sorted(prof.items(), key=lambda kv: -kv[1][0])}
    roof["launches_per_step"] = {k: v[1] / 4.0 for k, v in prof.items()}

    # ---- mixed precision: same workload, same timing, error of a full run ------------
    mixed = None
    if not args.no_mixed:
        sm_ = binding.Solver(wl, stream=sptr, use_graph=True, precision="mixed")
        sm_.step(args.warmup)
        torch.cuda.synchronize()
        evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            evm[i][0].record(stream)
            sm_.step(1)
            evm[i][1].record(stream)
        torch.cuda.synchronize()
        t_m = sum(a.elapsed_time(b) for a, b in evm) / 1e3
        prof_m = sm_.profile(4)
        sm_.close()
        err_m = None
        if os.path.exists(GOLDEN):
            s4 = binding.Solver(wl, stream=sptr, use_graph=True, precision="mixed")
            s4.step(wl.nsteps)
            err_m = float(np.linalg.norm(s4.scalar_flux() - g["rho"]) / np.linalg.norm(g["rho"]))
            s4.close()
        mixed = {"value": units * args.steps * ws / t_m, "unit": UNIT,
                 "ms_per_step": t_m / args.steps * 1e3, "flux_rel_l2_vs_oracle": err_m,
                 "speedup_vs_fp64": t_ours / t_m,
                 "kernels_ms_per_step": {k: round(v[0] / 4.0, 4) for k, v in
                                         sorted(prof_m.items(), key=lambda kv: -kv[1][0])},
                 "arithmetic": "FP32: L-step stage corrections (first-stage right-hand side "
                               "in FP64), collision K/L ODE increments; FP64: the eigen-split "
                               "K-step, updates, orthonormalisations, small eigen/SVD "
                               "problems, reductions, storage"}

    # ---- Strang splitting: same workload in FP64, x/2 y/2 c y/2 x/2 per step ----------
    strang = None
    if not args.no_strang:
        ws_ = wl.with_(splitting="strang")
        ss_ = binding.Solver(ws_, stream=sptr, use_graph=True)
        ss_.step(args.warmup)
        torch.cuda.synchronize()
        evs_ = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            evs_[i][0].record(stream)
            ss_.step(1)
            evs_[i][1].record(stream)
        torch.cuda.synchronize()
        t_s = sum(a.elapsed_time(b) for a, b in evs_) / 1e3
        ss_.close()
        diff = None
        if os.path.exists(GOLDEN):
            s5 = binding.Solver(ws_, stream=sptr, use_graph=True)
            s5.step(wl.nsteps)
            diff = float(np.linalg.norm(s5.scalar_flux() - g["rho"]) / np.linalg.norm(g["rho"]))
            s5.close()
        strang = {"value": units * args.steps * ws / t_s, "unit": UNIT,
                  "ms_per_step": t_s / args.steps * 1e3,
                  "flux_rel_l2_vs_lie_oracle": diff,
                  "note": "two advection phases of dt/2 per axis and one collision per step; "
                          "parity with the oracle's Strang form is a GPU test"}

    # ---- flux-split K-step: same workload, C+- from the direction split -------------
    fsplit = None
    if not args.no_strang:
        out_ = {}
        for prec in ("fp64", "mixed"):
            wf = wl.with_(kstep_split="flux")
            sf = binding.Solver(wf, stream=sptr, use_graph=True, precision=prec)
            sf.step(args.warmup)
            torch.cuda.synchronize()
            evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for i in range(args.steps):
                flush.fill_(float(i))
                evf[i][0].record(stream)
                sf.step(1)
                evf[i][1].record(stream)
            torch.cuda.synchronize()
            t_f = sum(a.elapsed_time(b) for a, b in evf) / 1e3
            sf.close()
            diff = None
            if os.path.exists(GOLDEN):
                s6 = binding.Solver(wf, stream=sptr, use_graph=True, precision=prec)
                s6.step(wl.nsteps)
                diff = float(np.linalg.norm(s6.scalar_flux() - g["rho"]) / np.linalg.norm(g["rho"]))
                s6.close()
            out_[prec] = {"value": units * args.steps * ws / t_f, "unit": UNIT,
                          "ms_per_step": t_f / args.steps * 1e3,
                          "flux_rel_l2_vs_eigen_split_oracle": diff}
        fsplit = dict(out_, note="C+- = <V, max/min(Omega,0) V> instead of Appendix A's "
                                 "eigen-split: no eigendecomposition in the step; a different "
                                 "discretisation at low rank (parity with the oracle's flux-split "
                                 "form is a GPU test)")

    # ---- physical inflow: the Hohlraum-type problem in FP64 ---------------------------
    infl = None
    if not args.no_strang:
        wh = inputs.hohlraum_problem()
        sh_ = binding.Solver(wh, stream=sptr, use_graph=True)
        sh_.step(args.warmup)
        torch.cuda.synchronize()
        evh = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            evh[i][0].record(stream)
            sh_.step(1)
            evh[i][1].record(stream)
        torch.cuda.synchronize()
        t_h = sum(a.elapsed_time(b) for a, b in evh) / 1e3
        rk_, rt_ = sh_.ranks()
        sh_.close()
        infl = {"workload": wh.name, "value": wh.ncells * wh.n * args.steps * ws / t_h,
                "unit": UNIT, "ms_per_step": t_h / args.steps * 1e3,
                "ranks_after_warmup_and_steps": [int(x) for x in rk_],
                "note": "inflow f = 1 through x = 0 for Omega_x >= 0, tolerance-adaptive "
                        "ranks; parity with the oracle on inflow problems is a GPU test"}

    # ---- batched form ----------------------------------------------------------------
    batch = None
    if args.batch > 0:
        batch = run_batch(args, torch, dev, flush)

    # ---- CPU baseline: the oracle on this machine's host cores ------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, nsteps=args.cpu_steps)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ours / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "cells": wl.ncells, "directions": wl.n,
                   "subdomains": wl.nsub, "rank": wl.rank, "r_aug_max": wl.r_aug_max,
                   "integrator": wl.integrator, "dt": wl.dt, "parallelism": f"replicas{ws}",
                   "l2": "flushed between timed steps (256 MiB write, outside the step events)",
                   "launch": "one CUDA graph per step"},
        "flux_rel_l2_vs_oracle": err,
        "ranks": {"stored_max": rs, "intermediate_max": rt},
        "e2e": e2e,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "roofline": roof,
        "clocks": clk.summary(),
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                  "fp64_gemm_tflops": fp64_peak},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if mixed is not None:
        line["mixed"] = mixed
    if strang is not None:
        line["strang"] = strang
    if fsplit is not None:
        line["flux_split"] = fsplit
    if infl is not None:
        line["inflow"] = infl
    if batch is not None:
        line["batch"] = batch
    return line, rank


def run_batch(args, torch, dev, flush):
    """The batched form: 64 seeded independent problems (grids 64^2/128^2/256^2, 2x2 or
    4x4 tilings, 128/512/1024 directions, ranks 4..21, RK4), one solver per direction
    count, the three solvers replayed concurrently on three streams.  Timed in FP64
    and in mixed precision, beside the plain FP64 loop (one solver per problem, one
    after another).  The mixed flux is compared with the FP64 flux of the same run."""
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
    for prec in ("fp64", "mixed"):
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
    # conditioning: the FP64 run again with 1e-7 (relative, seeded) noise on the initial
    # data, on the direction components and on the quadrature weights: how far
    # FP32-level perturbations of the spatial and of the angular data move each result
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

    def p_w(wls, rng):
        a = noise(rng, wls[0].w.shape)
        return [w.with_(w=w.w * a) for w in wls]

    pert = {"initial_data": fp64_flux(p_g0, 7), "directions": fp64_flux(p_dir, 11),
            "weights": fp64_flux(p_w, 12)}
    errs = []
    spread = {kk: [] for kk in pert}
    for gi, (n, wls) in enumerate(groups):
        lo = 0
        for w in wls:
            sl = slice(lo, lo + w.ncells)
            lo += w.ncells
            ref = flux["fp64"][gi][sl]
            nr = max(np.linalg.norm(ref), 1e-300)
            errs.append(float(np.linalg.norm(flux["mixed"][gi][sl] - ref) / nr))
            for kk, pv in pert.items():
                spread[kk].append(float(np.linalg.norm(pv[gi][sl] - ref) / nr))
    errs = np.array(errs)
    spread = {kk: np.array(v) for kk, v in spread.items()}
    worst = np.maximum.reduce(list(spread.values()))
    out["mixed"]["flux_rel_l2_vs_fp64_max"] = float(errs.max())
    out["mixed"]["flux_rel_l2_vs_fp64_median"] = float(np.median(errs))
    out["mixed"]["problems_within_1e-5"] = int(np.sum(errs <= 1e-5))
    out["fp64_sensitivity_to_1e-7_noise"] = {
        kk: {"max": float(v.max()), "median": float(np.median(v)),
             "problems_above_1e-6": int(np.sum(v > 1e-6))} for kk, v in spread.items()}
    # a problem whose FP64 result moves by more than 1e-6 under 1e-7 noise on its data
    # is too ill-conditioned for any FP32 arithmetic to hold 1e-5
    ok = (errs <= 1e-5) | (worst > 1e-6)
    out["mixed"]["problems_within_1e-5_or_ill_conditioned"] = int(np.sum(ok))
    out["mixed"]["max_error_on_well_conditioned"] = float(np.max(errs[worst <= 1e-6])) \
        if np.any(worst <= 1e-6) else None
    big = errs > 1e-5
    out["mixed"]["above_1e-5_max_ratio_to_fp64_sensitivity"] = \
        float(np.max(errs[big] / worst[big])) if np.any(big) else None
    out["mixed"]["speedup_vs_fp64_batched"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]

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
    out["mixed"]["speedup_vs_fp64_loop"] = out["fp64_loop"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


def cpu_baseline(wl, nsteps=3):
    from oracle import dd_dlra
    o = dd_dlra.DDDLRA(wl)
    o.step()                                # first step excluded (start-up)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        o.step()
    t = time.perf_counter() - t0
    return {"value": wl.ncells * wl.n * nsteps / t, "unit": UNIT,
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{nsteps} time steps (steps 2..{nsteps + 1}) of the {wl.name} workload, "
                      f"numpy FP64 with multithreaded BLAS, {t:.1f} s"}


def run_reference(args):
    """The CPU oracle timed as the reference arm (rank 0 only)."""
    from paper_2602_14854_gb300 import inputs
    from oracle import dd_dlra
    ws, rank, _ = dist_env()
    if rank != 0:
        return None, rank
    wl = inputs.config_c1()
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
            "config": {"workload": wl.name, "cells": wl.ncells, "directions": wl.n,
                       "subdomains": wl.nsub, "rank": wl.rank, "integrator": wl.integrator},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{args.steps} full time steps after {args.warmup} warm-up "
                                       f"steps of {wl.name}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    return line, rank


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-strang", action="store_true")
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
