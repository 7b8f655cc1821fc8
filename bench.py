"""Benchmark: fused SSP-RK2 finite-volume step of the level-2 shallow-moment model on a
2048 x 2048 structured grid (7 variables, FP32 state), one JSON line on rank 0.

Workload (seeded, synthetic): Gaussian surface bump (amplitude U[0.1, 0.5], sigma 0.05) on a
lake of level 1 over an 8-mode Fourier bathymetry of amplitude 0.2, wall boundaries, Navier slip
C = 0.1 with Newtonian nu = 0.01, adaptive CFL 0.45 step computed on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm) on the host cores on a bounded
window of the same workload.  For N > 1 (torchrun) every rank runs an independent replica of the
workload (one grid is not split across GPUs): weak scaling.

Other workloads print their own lines: --workload tri | ensemble | closure | closure-kernels |
dambreak1d | lift | vam.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 2048
LEVEL = 2
NV = 2 * LEVEL + 3
FRIC = dict(kind=1, C=0.1, nu=0.01)
CFL = 0.45
# algorithmic bytes per cell and launch (FP32): stage 1 reads Q^n (7) + b, writes Q1 (7);
# stage 2 reads Q1 (7) + b + Q^n (7), writes Q^{n+1} (7)
BYTES_STAGE = {1: 4 * (NV + 1 + NV), 2: 4 * (NV + 1 + NV + NV)}
METRIC = "cell-updates/sec and % of HBM peak per FV step"
KERNEL_SOURCES = ["paper_2601_04826_gb300/csrc/fv_struct2d_f32.cu", "paper_2601_04826_gb300/csrc/struct2d_f32.cuh",
                  "paper_2601_04826_gb300/csrc/f32x2.cuh",
                  "paper_2601_04826_gb300/csrc/model.cuh", "paper_2601_04826_gb300/csrc/fv_common.cuh",
                  "paper_2601_04826_gb300/csrc/basis.cuh"]


TRI_KERNEL_SOURCES = ["paper_2601_04826_gb300/csrc/fv_tri.cu", "paper_2601_04826_gb300/csrc/model.cuh",
                      "paper_2601_04826_gb300/csrc/fv_common.cuh", "paper_2601_04826_gb300/csrc/basis.cuh"]


def kernel_hash(sources=None):
    h = hashlib.sha256()
    for p in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(sources=None):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary, if it was taken on the
    current source of that kernel (the summary line carries a hash of the kernel's source files)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    want = kernel_hash(sources)
    for fn in sorted(os.listdir(d)):
        if not fn.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(d, fn)):
            m = re.search(r"traffic_per_launch_bytes:\s*([0-9.eE+]+)\s+source_hash:\s*([0-9a-f]+)", line)
            if m and m.group(2) == want:
                return float(m.group(1))
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def peaks_tensor():
    """Dense BF16 tensor peak in TFLOP/s: the measured sustained cuBLAS figure (a kernel timed inside a
    long run), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        v = d.get("bf16_tflops_sustained") or d.get("bf16_tflops")
        if v:
            return float(v), "measured sustained" if d.get("bf16_tflops_sustained") else "measured burst"
    return 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        loaded = [s for s, _, _ in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(m for _, m, _ in rows),
                "reasons": reasons, "samples": len(rows)}


def workload():
    from paper_2601_04826_gb300 import inputs

    Q0, b = inputs.gaussian_bump_2d(N_SIDE, N_SIDE, LEVEL, seed=0)
    return Q0, b


def max_over_ranks(x, world, device):
    """The maximum of a per-rank float over all ranks (the slowest replica times the job)."""
    if world <= 1:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, seconds_max, world):
    """Whole-job throughput of independent replicas: the units all ranks advanced over the slowest
    rank's time (weak scaling: every rank advances the same workload)."""
    return world * units_per_rank * steps / seconds_max


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2601_04826_gb300 import build, zoomy

    if rank == 0 or not os.path.exists(zoomy.LIB_PATH):
        build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    Q0, b = workload()
    nc = N_SIDE * N_SIDE
    fr = zoomy.friction(FRIC["kind"], C=FRIC["C"], nu=FRIC["nu"])
    ctx = zoomy.Context(zoomy.mesh_2d(N_SIDE, N_SIDE, bathymetry=b), LEVEL, fr, cfl=CFL, dtype=zoomy.FP32)
    Q = torch.tensor(Q0, dtype=torch.float32, device=dev)

    if args.order == 2:
        zoomy.zoomy_space_order(ctx.ctx, 2)
    # launch configuration from the autotuner (or given, for profiling runs), then warm-up
    if args.order == 2:
        tuned_rows = None  # the second-order kernel is cell-centric
    elif args.rows_per_warp:
        zoomy.zoomy_tune_set(ctx.ctx, args.rows_per_warp, 1)
        tuned_rows = args.rows_per_warp
    else:
        tuned_rows, _ = ctx.autotune(Q)
    ctx.step(Q, nsteps=args.warmup, dt=0.0)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.step(Q, nsteps=args.steps, dt=0.0, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    t_sim = zoomy.zoomy_sync(ctx.ctx)  # raises on a device-detected error
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    # per-kernel launch durations: the same steps again with CUDA events around every stage launch on
    # the library's stream (an event between two launches ends their programmatic overlap, so the
    # timed region above runs without them)
    nprof = min(args.steps, 500)
    zoomy.zoomy_profile_enable(ctx.ctx, True)
    ctx.step(Q, nsteps=nprof, dt=0.0, sync=False)
    zoomy.zoomy_sync(ctx.ctx)
    launches, kms = zoomy.zoomy_profile_read(ctx.ctx)
    zoomy.zoomy_profile_enable(ctx.ctx, False)

    # end-to-end through the host-buffer entry point: H2D of the state, one step, D2H of the result
    e2e_s = float("nan")
    if not args.no_e2e:
        Qh = torch.tensor(Q0, dtype=torch.float32).pin_memory()
        ctx.step_host(Qh, nsteps=1, dt=0.0)
        n_e2e = max(3, min(args.steps, 30))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            ctx.step_host(Qh, nsteps=1, dt=0.0)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / n_e2e, world, dev)
    ctx.close()

    if rank != 0:
        return None
    hbm, peak_kind = peaks()
    avg2 = kms[1] / max(launches[1], 1)
    avg1 = kms[0] / max(launches[0], 1)
    dom = 2 if avg2 >= avg1 else 1
    avg = avg2 if dom == 2 else avg1
    achieved = BYTES_STAGE[dom] * nc / (avg * 1e-3) / 1e9
    traffic = ncu_traffic() if dom == 2 and args.order == 1 else None
    kname = f"k_stage_2d_f32<2,{dom}>" if args.order == 1 else f"k_stage_order2_march<2,float,{dom}>"
    value = job_throughput(nc, args.steps, ms * 1e-3, world)
    step_bytes = (BYTES_STAGE[1] + BYTES_STAGE[2]) * nc
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "cell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Gaussian bump over 8-mode Fourier bathymetry)",
        "config": {"workload": "2D shallow-moment level 2, 2048x2048 structured grid, 7 vars, FP32 state, walls, "
                               "slip C=0.1 + Newtonian nu=0.01, SSP-RK2, adaptive CFL 0.45",
                   "cells": nc, "level": LEVEL, "global_batch": world, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (Q 117 MB + stage buffer 117 MB + bed 17 MB per replica)",
                   "step_hbm_fraction": step_bytes / (ms / args.steps * 1e-3) / 1e9 / hbm,
                   "rows_per_warp": tuned_rows,
                   "space_order": args.order,
                   "sim_time_advanced": t_sim},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                     "algorithmic_bytes_per_launch": BYTES_STAGE[dom] * nc,
                     "avg_launch_ms": {"stage1": avg1, "stage2": avg2}},
        "e2e": None if args.no_e2e else {"value": job_throughput(nc, 1, e2e_s, world), "unit": "cell-updates/s",
                                         "h2d_bytes_per_step": 4 * NV * nc, "d2h_bytes_per_step": 4 * NV * nc},
        "gpu_launches": int(2 * args.steps + 1),
        "clocks": clk.summary(),
    }
    line["roofline"]["launch_timing"] = (f"CUDA events around each stage launch, {nprof} steps right after the "
                                         "timed region (same state, same launch configuration)")
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    return line


def run_tri(args):
    """Config-3 workload: ~4M-triangle jittered Delaunay mesh, level 3, Manning, circular dam break into a
    dry domain, walls.  Prints its own JSON line (not the default bench line)."""
    import numpy as np
    import torch

    from paper_2601_04826_gb300 import build, inputs, zoomy

    build.build()
    level, nv = 3, 9
    verts, tris = inputs.jittered_delaunay(args.tri_side, seed=0)
    Q0 = inputs.circular_dam_tri(verts, tris, level, radius=0.2, h_in=1.5)
    nc = len(tris)
    ctx = zoomy.Context(zoomy.mesh_tri(verts, tris, bc=1), level, zoomy.friction(2, manning_n=0.03), dtype=0)
    perm = ctx.permutation()
    Q = torch.tensor(np.ascontiguousarray(Q0[:, perm]), dtype=torch.float32, device="cuda")
    ctx.step(Q, nsteps=args.warmup, dt=0.0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.step(Q, nsteps=args.steps, dt=0.0, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
    zoomy.zoomy_sync(ctx.ctx)
    ms = e0.elapsed_time(e1)
    # per-kernel durations from a second pass with events around every launch (they end the
    # programmatic overlap of consecutive launches, so the timed pass runs without them)
    zoomy.zoomy_profile_enable(ctx.ctx, True)
    ctx.step(Q, nsteps=min(args.steps, 200), dt=0.0)
    launches, kms = zoomy.zoomy_profile_read(ctx.ctx)
    ctx.close()
    hbm, peak_kind = peaks()
    # per cell: state nv, bed, geometry (3 neighbours int32 + 3 normals + 3 |e|/|Omega| as float32) read once,
    # state written; stage 2 also reads Q^n
    geo = 4 * 12
    b1, b2 = 4 * (nv + 1 + nv) + geo, 4 * (nv + 1 + nv + nv) + geo
    avg2 = kms[1] / max(launches[1], 1)
    ach = b2 * nc / (avg2 * 1e-3) / 1e9
    return {"metric": METRIC, "value": nc * args.steps / (ms * 1e-3), "unit": "cell-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded jittered Delaunay)",
            "config": {"workload": "2D shallow-moment level 3 on a jittered-point Delaunay triangle mesh "
                                   f"({nc} cells, Morton order), Manning n=0.03, dry outside a circular dam, walls"},
            "roofline": {"bound": "hbm", "kernel": "k_stage_tri<3,2>", "achieved": ach, "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / hbm,
                         "traffic": ncu_traffic(TRI_KERNEL_SOURCES) if args.tri_side == 1415 else None,
                         "algorithmic_bytes_per_launch": b2 * nc,
                         "avg_launch_ms": {"stage1": kms[0] / max(launches[0], 1), "stage2": avg2},
                         "launch_timing": "CUDA events around each launch in a second pass after the timed one"},
            "gpu_launches": int(2 * args.steps + 1), "clocks": clk.summary()}


def run_ensemble(args):
    """Config-4 workload: 512 independent level-1 members, sides ~ U{64..512}, slip ~ logNormal(-2, 0.5),
    one persistent launch per call captured in a CUDA graph.  Prints its own JSON line."""
    import torch

    from paper_2601_04826_gb300 import build, inputs, zoomy

    build.build()
    level, nv = 1, 5
    sides, slip, seeds = inputs.ensemble_members(512, seed=0)
    Q0, offs = inputs.ensemble_state(sides, seeds, level)
    nc = int(offs[-1])
    ens = zoomy.zoomy_ensemble_create(sides, slip, level)
    Q = torch.tensor(Q0, dtype=torch.float32, device="cuda")
    rows, _ = zoomy.zoomy_ensemble_autotune(ens, Q, nc)
    zoomy.zoomy_ensemble_step(ens, Q, nc, args.warmup, mode=0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        zoomy.zoomy_ensemble_step(ens, Q, nc, args.steps, mode=0)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    zoomy.zoomy_mesh_destroy(ens)
    hbm, peak_kind = peaks()
    step_bytes = 4 * ((nv + 1 + nv) + (3 * nv + 1)) * nc  # both stages, bed included
    achieved = step_bytes * args.steps / (ms * 1e-3) / 1e9
    return {"metric": METRIC, "value": nc * args.steps / (ms * 1e-3), "unit": "cell-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded Gaussian bumps)",
            "config": {"workload": f"batched ensemble: 512 level-1 members, sides U{{64..512}} ({nc} cells), "
                                   "slip logNormal(-2, 0.5), walls, one persistent cooperative launch per call in "
                                   "a CUDA graph", "rows_per_warp": rows},
            "roofline": {"bound": "hbm", "kernel": "k_ensemble_persistent<1>", "achieved": achieved, "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "note": "whole persistent launch (both stages and barriers) over its duration"},
            "gpu_launches": 1, "clocks": clk.summary()}


def run_closure_kernels(args):
    """The closed level-1 step alone on the 1024^2 closure workload with an untrained (Glorot) network:
    per-kernel launch times of the prediction and stage kernels, for profiling runs.  Prints its own
    JSON line (no training, no level-4 comparison)."""
    import numpy as np
    import torch

    from paper_2601_04826_gb300 import build, closure, inputs, zoomy

    build.build()
    side = 1024
    _, lam, seeds = inputs.ensemble_members(1, seed=4242)
    params = closure.init_params(0)
    ins = np.array([1.0, 4.0, 4.0, 50.0, 50.0, 4.0])
    outs = np.full(6, 1e-3)
    r = closure.Run(side, 1, float(lam[0]), int(seeds[0]), closure=(params, ins, outs),
                    schedule=args.closure_schedule)
    zoomy.zoomy_closure_engine(r.ctx.ctx, args.closure_engine)
    r.ctx.step(r.Q, nsteps=args.warmup, dt=0.0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r.ctx.step(r.Q, nsteps=args.steps, dt=0.0, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    zoomy.zoomy_sync(r.ctx.ctx)
    ms = e0.elapsed_time(e1)
    # per-kernel durations in a second pass with events around every launch (they end the
    # programmatic overlap of consecutive launches, so the timed pass runs without them)
    zoomy.zoomy_profile_enable(r.ctx.ctx, True)
    r.ctx.step(r.Q, nsteps=args.steps, dt=0.0, sync=False)
    zoomy.zoomy_sync(r.ctx.ctx)
    launches, kms = zoomy.zoomy_profile_read(r.ctx.ctx)
    r.close()
    flop_eval = 2 * (6 * 64 + 64 * 64 + 64 * 6)
    avg = [kms[i] / max(launches[i], 1) for i in range(3)]
    return {"metric": "closed level-1 step time", "value": ms / args.steps, "unit": "ms/step", "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False,
            "config": {"workload": f"learned-closure step kernels, {side}x{side}, untrained network",
                       "engine": ["tcgen05", "mma.sync"][args.closure_engine],
                       "schedule": ["every stage", "once per step"][args.closure_schedule]},
            "avg_launch_ms": {"stage1": avg[0], "stage2": avg[1], "predict": avg[2]},
            "predict_tflops": flop_eval * side * side / (avg[2] * 1e-3) / 1e12, "gpu_launches": int(sum(launches)),
            "launch_timing": "per-kernel averages from a second pass with CUDA events around every launch"}


def run_closure(args):
    """Config-5 workload: train the closure on seeded level-4 runs, then time-to-solution at T = 2 on a
    1024^2 held-out member: plain level 4 against level 1 closed by the network (and plain level 1),
    with the relative L1 errors of (h, h u_m, h v_m) against level 4.  Prints its own JSON line."""
    import time

    import numpy as np
    import torch

    from paper_2601_04826_gb300 import build, closure, inputs, zoomy

    build.build()
    T, side = 2.0, 1024
    t0 = time.perf_counter()
    F, Y, _ = closure.generate_samples(nmembers=args.closure_members, side=args.closure_train_side, level=4, T=T,
                                       snapshots=8, seed=3)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    ins, outs = closure.scales(F, Y)
    t0 = time.perf_counter()
    params, hist = closure.fit(F, Y, ins, outs, steps=3000, batch=16384, seed=0)
    t_train = time.perf_counter() - t0
    nsamples = int(F.shape[0])
    del F, Y
    torch.cuda.empty_cache()
    _, lam, seeds = inputs.ensemble_members(1, seed=4242)
    lam, seed = float(lam[0]), int(seeds[0])
    res = {}
    with ClockSampler(0) as clk:
        for name, lv, cl, sched in (("level4", 4, None, 0), ("closure", 1, (params, ins, outs), 1),
                                    ("closure_every_stage", 1, (params, ins, outs), 0), ("level1", 1, None, 0)):
            r = closure.Run(side, lv, lam, seed, closure=cl, schedule=sched)
            if cl is None:
                r.ctx.autotune(r.Q)
            r.ctx.step(r.Q, nsteps=3, dt=1e-6)  # warm-up (module load, first launches)
            r.Q.copy_(closure.Run.initial(side, lv, seed))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nsteps = r.run_to(T)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            state = r.mean_state()
            # per-kernel durations: 100 more steps with CUDA events around every launch (not timed above:
            # the events end the programmatic overlap of consecutive launches)
            zoomy.zoomy_profile_enable(r.ctx.ctx, True)
            r.ctx.step(r.Q, nsteps=100, dt=1e-5)
            launches, kms = zoomy.zoomy_profile_read(r.ctx.ctx)
            res[name] = {"time_s": wall, "steps": nsteps, "state": state,
                         "kernel_ms": [kms[i] / max(launches[i], 1) for i in range(3)],
                         "launches": int(sum(launches))}
            r.close()
    ref = res["level4"]["state"]

    def l1(st):
        return [float(v) for v in np.abs(st - ref).sum(axis=1) / np.abs(ref).sum(axis=1)]

    cl_, l4 = res["closure"], res["level4"]
    # tensor work of one prediction launch: one network evaluation per cell
    flop_eval = 2 * (6 * 64 + 64 * 64 + 64 * 6)
    cells = side * side
    ach = flop_eval * cells / (cl_["kernel_ms"][2] * 1e-3) / 1e12
    pk = peaks_tensor()
    return {"metric": "time_to_solution", "value": cl_["time_s"], "unit": "s", "n_gpus": 1, "steps": cl_["steps"],
            "warmup": 3, "ms_per_step": 1e3 * cl_["time_s"] / cl_["steps"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic (seeded Gaussian bumps)",
            "config": {"workload": f"learned closure: level 1 + MLP on {side}x{side}, walls, T={T}, slip "
                                   f"{lam:.4f} (held-out member), vs plain level 4",
                       "training": {"members": args.closure_members, "side": args.closure_train_side,
                                    "samples": nsamples, "adam_steps": 3000, "batch": 16384,
                                    "data_s": t_data, "train_s": t_train, "loss": hist[-1][1]}},
            "level4": {"time_s": l4["time_s"], "steps": l4["steps"], "ms_per_step": 1e3 * l4["time_s"] / l4["steps"]},
            "level1": {"time_s": res["level1"]["time_s"], "steps": res["level1"]["steps"]},
            "closure_every_stage": {"time_s": res["closure_every_stage"]["time_s"],
                                    "steps": res["closure_every_stage"]["steps"],
                                    "speedup_vs_level4": l4["time_s"] / res["closure_every_stage"]["time_s"]},
            "speedup_vs_level4": l4["time_s"] / cl_["time_s"],
            "closure_schedule": "once per step (network on Q^n, held for both stages)",
            "rel_l1_vs_level4": {"closure": l1(cl_["state"]), "closure_every_stage": l1(res["closure_every_stage"]["state"]),
                                 "level1": l1(res["level1"]["state"]), "vars": ["h", "h u_m", "h v_m"]},
            "roofline": {"bound": "tensor", "kernel": "k_closure_predict", "achieved": ach, "peak": pk[0],
                         "peak_kind": pk[1], "unit": "TFLOP/s", "frac": ach / pk[0], "traffic": None,
                         "algorithmic_flop_per_launch": flop_eval * cells,
                         "avg_launch_ms": {"predict": cl_["kernel_ms"][2], "stage1": cl_["kernel_ms"][0],
                                           "stage2": cl_["kernel_ms"][1]},
                         "note": "network FLOPs (unpadded 6-64-64-6) of one prediction launch over its average "
                                 "duration; BF16 operands, FP32 accumulation"},
            "gpu_launches": int(cl_["launches"]), "clocks": clk.summary()}


def _dambreak1d_time(zoomy, Q0, nx, level, steps, warmup, mode, wpc):
    """us per step of one zoomy_step call of `steps` CFL steps (after `warmup` steps) in launch shape
    (mode, warps per CTA); returns (us, simulated time advanced)."""
    import torch

    ctx = zoomy.Context(zoomy.mesh_1d(nx, 0.0, 10.0, bc=(0, 0)), level,
                        zoomy.friction(zoomy.FRICTION_SLIP_NEWTONIAN, C=0.1, nu=0.01), cfl=0.45, dtype=zoomy.FP64)
    ctx.tune_1d(mode, wpc)
    Q = torch.tensor(Q0, dtype=torch.float64, device="cuda")
    ctx.step(Q, nsteps=warmup, dt=0.0)
    Q.copy_(torch.tensor(Q0, dtype=torch.float64))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(Q, nsteps=steps, dt=0.0, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t = zoomy.zoomy_sync(ctx.ctx)
    ms = e0.elapsed_time(e1)
    ctx.close()
    return 1e3 * ms / steps, t


def run_dambreak1d(args):
    """The 1D dam break (2000 cells, level 1, FP64, slip + Newtonian, transmissive): a latency-bound
    case (the whole state is 48 KB), reported as time per step in the automatic launch shape (two
    launches per step, one-warp CTAs), with other launch shapes (zoomy_tune_1d) timed beside it.
    Prints its own JSON line."""
    from paper_2601_04826_gb300 import build, inputs, zoomy

    build.build()
    nx, level = 2000, 1
    Q0 = inputs.dambreak_1d(nx, 0.0, 10.0, h_left=2.0, h_right=1.0, x_dam=5.0, level=level)
    us, t = _dambreak1d_time(zoomy, Q0, nx, level, args.steps, args.warmup, zoomy.LAUNCH_AUTO, 0)
    shapes = {}
    for name, mode, wpc in [("per_stage_1warp", zoomy.LAUNCH_PER_STAGE, 1), ("per_stage_2warps", zoomy.LAUNCH_PER_STAGE, 2),
                            ("persistent_1warp", zoomy.LAUNCH_PERSISTENT, 1)]:
        shapes[name] = round(_dambreak1d_time(zoomy, Q0, nx, level, args.steps, args.warmup, mode, wpc)[0], 3)
    return {"metric": "time per SSP-RK2 step", "value": us, "unit": "us/step",
            "cell_updates_per_s": nx * 1e6 / us, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1D shallow-moment level 1 dam break, 2000 cells on [0,10], h = 2 / 1, slip "
                                   "C=0.1 + Newtonian nu=0.01, transmissive, adaptive CFL 0.45",
                       "sim_time_advanced": t},
            "launch_shapes_us_per_step": shapes,
            "gpu_launches": 2 * args.steps + 1}


def run_lift(args):
    """Lifting of the 2048^2 level-2 bench state to K = 16 sigma levels (u, v, w, p: 1.07 GB written per
    launch).  Prints its own JSON line."""
    import numpy as np
    import torch

    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    Q0, b = workload()
    nc, K = N_SIDE * N_SIDE, 16
    fr = zoomy.friction(FRIC["kind"], C=FRIC["C"], nu=FRIC["nu"])
    ctx = zoomy.Context(zoomy.mesh_2d(N_SIDE, N_SIDE, bathymetry=b), LEVEL, fr, cfl=CFL, dtype=zoomy.FP32)
    Q = torch.tensor(Q0, dtype=torch.float32, device="cuda")
    ctx.step(Q, nsteps=50, dt=0.0)  # a state with moving water
    zeta = (np.arange(K) + 0.5) / K
    out = torch.empty((4 * K, nc), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        zoomy.zoomy_lift3d(ctx.ctx, Q, nc, zeta, out, nc)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            zoomy.zoomy_lift3d(ctx.ctx, Q, nc, zeta, out, nc)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ctx.close()
    hbm, peak_kind = peaks()
    per_cell = 4 * (NV + 1) + 4 * 4 * K  # state + bed read once, four fields at K levels written
    ach = per_cell * nc / (ms * 1e-3) / 1e9
    return {"metric": "lifted cells/s", "value": nc / (ms * 1e-3), "unit": "cells/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (bench state after 50 steps)",
            "config": {"workload": f"lifting of the 2048x2048 level-2 state to u, v, w, p at {K} sigma levels"},
            "roofline": {"bound": "hbm", "kernel": "k_lift3d<2,1,float>", "achieved": ach, "peak": hbm,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                         "algorithmic_bytes_per_launch": per_cell * nc},
            "gpu_launches": args.steps, "clocks": clk.summary()}


def vam_launches_per_step(n, cr=2):
    """Wave speed, predictor, assembly, correction, the block inversion, cr cyclic-reduction levels, the
    parallel levels of the remaining system and cr back-substitutions (N = ceil(n / 2) block rows), as the
    library launches them."""
    N = (n + 1) // 2
    sr, k = 1, 0
    while k < cr and 2 * sr < N:
        sr, k = 2 * sr, k + 1
    levels, s = 0, sr
    while s < N:
        levels, s = levels + 1, 2 * s
    return 5 + k + levels + k


def run_vam(args):
    """The VAM predictor-corrector in 1D: a small solitary-like hump on depth 1 (2000 cells on [0, 20],
    walls, FP64), time per step (wave-speed reduction, predictor, block-tridiagonal pressure assembly,
    cyclic-reduction levels, corrector).  Prints its own JSON line."""
    import numpy as np
    import torch

    from paper_2601_04826_gb300 import build, zoomy

    build.build()
    n, L = 2000, 20.0
    x = (np.arange(n) + 0.5) * L / n
    Q0 = np.zeros((5, n))
    Q0[0] = 1.0 + 0.2 / np.cosh(np.sqrt(0.75 * 0.2) * (x - 5.0)) ** 2
    Q0[1] = Q0[0] * np.sqrt(9.81 * 1.2) * (1.0 - 1.0 / Q0[0])
    ctx = zoomy.Context(zoomy.mesh_1d(n, 0.0, L, bc=(1, 1)), 1, zoomy.friction(0), cfl=0.45, dtype=zoomy.FP64)
    ctx.vam(True)
    Q = torch.tensor(Q0, dtype=torch.float64, device="cuda")
    ctx.step(Q, nsteps=args.warmup, dt=0.0)
    Q.copy_(torch.tensor(Q0, dtype=torch.float64))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(Q, nsteps=args.steps, dt=0.0, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t = zoomy.zoomy_sync(ctx.ctx)
    ms = e0.elapsed_time(e1)
    ctx.close()
    return {"metric": "time per VAM predictor-corrector step", "value": 1e3 * ms / args.steps, "unit": "us/step",
            "cell_updates_per_s": n * args.steps / (ms * 1e-3), "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1D non-hydrostatic VAM, 2000 cells on [0,20], depth 1 with a 0.2 hump, walls, "
                                   "adaptive CFL 0.45", "sim_time_advanced": t},
            "gpu_launches": vam_launches_per_step(n) * args.steps}


def oracle_window_run(side, nsteps):
    """The oracle on a side x side window of the workload (cells of the 2048^2 grid, walls)."""
    import numpy as np

    from oracle import oracle as O

    Q0, b = workload()
    Q0 = Q0.astype(np.float32).astype(np.float64)
    b = b.astype(np.float32).astype(np.float64)
    if side < N_SIDE:
        # window centred on the bump's centre region
        j0 = i0 = (N_SIDE - side) // 2
        idx = (np.arange(j0, j0 + side)[:, None] * N_SIDE + np.arange(i0, i0 + side)[None, :]).reshape(-1)
        Q0 = Q0[:, idx]
        b = b[idx]
    h = 1.0 / N_SIDE
    md = O.Model(LEVEL, 2, g=9.81, h_dry=1e-6, friction=FRIC["kind"], C=FRIC["C"], nu=FRIC["nu"])
    mesh = O.Mesh.rect(side, side, 0, side * h, 0, side * h, bc=(1, 1, 1, 1))
    t0 = time.perf_counter()
    O.step(md, mesh, Q0, nsteps, dt=0.0, cfl=CFL, bed=b)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args):
    side, nsteps = N_SIDE, 2
    secs = oracle_window_run(side, nsteps)
    threads = int(os.environ.get("OMP_NUM_THREADS", host_cores()))
    return {"value": side * side * nsteps / secs, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
            "sample": f"{nsteps} SSP-RK2 steps of the full {side}x{side} level-2 workload, FP64 C oracle, OpenMP "
                      f"over cells, {secs:.1f} s"}


def run_side_workloads(args):
    """The other workloads, timed after the headline in the same run (shorter: fewer steps), each summarised
    by its metric, time per step and the roofline fraction of its dominant kernel.  A workload that fails
    is reported with its error and does not affect the headline."""
    import argparse as _ap

    import torch

    runs = [("order2_2048_level2", run_ours, dict(order=2, steps=200, warmup=5, no_cpu_baseline=True, no_e2e=True)),
            ("dambreak1d_2000_fp64", run_dambreak1d, dict(steps=400, warmup=5)),
            ("vam1d_2000_fp64", run_vam, dict(steps=200, warmup=5)),
            ("lift3d_2048_level2_k16", run_lift, dict(steps=20, warmup=3)),
            ("ensemble_512_level1", run_ensemble, dict(steps=50, warmup=3)),
            ("triangles_4m_level3", run_tri, dict(steps=100, warmup=5, tri_side=1415)),
            ("closure_1024_to_T2", run_closure, dict(steps=1, warmup=3))]
    out = {}
    for name, fn, kw in runs:
        a = _ap.Namespace(**vars(args))
        for k, v in kw.items():
            setattr(a, k, v)
        t0 = time.perf_counter()
        try:
            line = fn(a, 0, 1, 0) if fn is run_ours else fn(a)
            rf = line.get("roofline") or {}
            out[name] = {"metric": line.get("metric"), "value": line.get("value"), "unit": line.get("unit"),
                         "ms_per_step": line.get("ms_per_step"), "kernel": rf.get("kernel"), "frac": rf.get("frac"),
                         "clocks": line.get("clocks"), "wall_s": round(time.perf_counter() - t0, 1)}
            for extra in ("launch_shapes_us_per_step", "variants_ms_per_step", "speedup_vs_level4", "level4",
                          "rel_l1_vs_level4"):
                if extra in line:
                    out[name][extra] = line[extra]
        except Exception as e:  # noqa: BLE001 -- reported in the line, the headline stands
            out[name] = {"error": f"{type(e).__name__}: {str(e)[:200]}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    # window sized so that warmup + steps end within about two minutes
    probe_side = 256
    t = oracle_window_run(probe_side, 1)
    per_cell = t / (probe_side * probe_side)
    budget = 110.0
    cells = budget / max(args.steps + args.warmup, 1) / per_cell
    side = int(max(32, min(N_SIDE, cells ** 0.5)))
    if args.warmup:
        oracle_window_run(side, args.warmup)
    t0 = time.perf_counter()
    oracle_window_run(side, args.steps)
    secs = time.perf_counter() - t0
    value = side * side * args.steps / secs
    threads = int(os.environ.get("OMP_NUM_THREADS", host_cores()))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian bump over 8-mode Fourier bathymetry)",
            "config": {"workload": "2D shallow-moment level 2, 2048x2048 structured grid, 7 vars, walls, "
                                   "slip C=0.1 + Newtonian nu=0.01, SSP-RK2, adaptive CFL 0.45",
                       "window": f"{side}x{side} cells of the 2048^2 workload per step"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
                             "sample": f"{side}x{side} window, {args.steps} SSP-RK2 steps"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--workload", choices=["grid", "tri", "ensemble", "closure", "closure-kernels", "dambreak1d",
                                           "lift", "vam"],
                    default="grid",
                    help="grid: the 2048^2 level-2 benchmark (default); tri: the ~4M-triangle level-3 dam break; "
                         "ensemble: 512 ragged level-1 members in one persistent launch; closure: learned "
                         "closure vs level 4, time to T = 2 on 1024^2")
    ap.add_argument("--closure-members", type=int, default=256, help="level-4 training runs (closure workload)")
    ap.add_argument("--order", type=int, choices=[1, 2], default=1,
                    help="space order of the grid workload (1: the benchmark scheme; 2: MUSCL)")
    ap.add_argument("--tri-side", type=int, default=1415,
                    help="lattice side of the triangle workload (1415: ~4M triangles; smaller for profiling runs)")
    ap.add_argument("--closure-train-side", type=int, default=128, help="grid side of the training runs")
    ap.add_argument("--closure-engine", type=int, default=0, help="closure network engine: 0 tcgen05, 1 mma.sync")
    ap.add_argument("--closure-schedule", type=int, default=1, choices=[0, 1],
                    help="closure-kernels: network on every stage input (0) or once per step (1)")
    ap.add_argument("--no-side", action="store_true",
                    help="grid workload: skip the shorter runs of the other workloads after the headline")
    ap.add_argument("--rows-per-warp", type=int, default=0,
                    help="fixed structured-kernel segment height instead of the autotuner (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    elif args.workload == "tri":
        line = run_tri(args) if rank == 0 else None
    elif args.workload == "ensemble":
        line = run_ensemble(args) if rank == 0 else None
    elif args.workload == "closure":
        line = run_closure(args) if rank == 0 else None
    elif args.workload == "closure-kernels":
        line = run_closure_kernels(args) if rank == 0 else None
    elif args.workload == "dambreak1d":
        line = run_dambreak1d(args) if rank == 0 else None
    elif args.workload == "lift":
        line = run_lift(args) if rank == 0 else None
    elif args.workload == "vam":
        line = run_vam(args) if rank == 0 else None
    else:
        line = run_ours(args, rank, world, local_rank)
        if line is not None and world == 1 and args.order == 1 and not args.no_side:
            line["side_workloads"] = run_side_workloads(args)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl == "ours":
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
