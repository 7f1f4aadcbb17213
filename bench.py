#!/usr/bin/env python3
"""Throughput of the coupled EM-thermal-mechanical hot path on the full-scale
1024 x 1024 x 128 voxel package (134 M cells, FP32 fields, FP64 reductions).

One step = one pass of every stage of the path over the package:
  EM burst slice (N_EM leapfrog steps, Joule accumulation fused)
  -> burst-averaged Joule source -> N_TH forward-Euler thermal steps
  -> thermoelastic solve slice (thermal load, Jacobi diagonal, N_CG PCG
     iterations, von Mises and |u|).
The slice sizes keep the full job's proportions (2 ns burst = 314,701 EM
steps : 10^4 thermal steps : one solve of ~10^4 CG iterations, scaled by
about 1/3300). value = EM + thermal grid-point updates (EM cell-steps +
thermal node-steps) per second of the whole step, the stress slice's time
included: the job's EM+thermal throughput. The stress solve is reported on
its own (stress_cg: a whole FP32-in-FP64-refinement solve of the package to
a 1e-9 relative residual, s/solve).

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank solves its own package (replicas, no collective on
the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EM, N_TH, N_CG = 96, 3, 3
N_CPL = 32  # coupled EM + thermal steps timed after the main region
METRIC = "Gcell-updates/s & % HBM roofline (EM+thermal); stress-CG s/solve; designs/hr, p50/p99"
UNIT = "Gcell-updates/s"
def workload_name(nx, ny, nz=128):
    """The workload label: the full-scale package at the default size, else
    the reduced grid that was actually run."""
    if (nx, ny, nz) == (1024, 1024, 128):
        return "full-scale layered package 1024x1024x128 (134M cells), FP32"
    return f"layered package {nx}x{ny}x{nz} ({nx * ny * nz / 1e6:.0f}M cells, reduced), FP32"


def parse():
    a = argparse.ArgumentParser()
    a.add_argument("--gpus", type=int, default=1)
    a.add_argument("--steps", type=int, default=5)
    a.add_argument("--warmup", type=int, default=3)
    a.add_argument("--impl", default="cosim", choices=["cosim", "reference"])
    a.add_argument("--nx", type=int, default=1024)
    a.add_argument("--ny", type=int, default=1024)
    a.add_argument("--nz", type=int, default=128, help="layers of the package (>= 64; reduced grids for profiling)")
    a.add_argument("--no-e2e", action="store_true")
    a.add_argument("--no-cpu", action="store_true")
    a.add_argument("--no-serve", action="store_true")
    a.add_argument("--no-batch", action="store_true")
    a.add_argument("--no-cg-solve", action="store_true")
    a.add_argument("--serve-n", type=int, default=16)
    a.add_argument("--serve-em-steps", type=int, default=512)
    a.add_argument("--serve-config5", action="store_true",
                   help="only the serving trace of the full design mix with 10%% full-scale packages "
                        "(several minutes); prints its JSON object")
    return a.parse_args()


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm

def em_alg_bytes(ctx, p):
    """algorithmic HBM bytes of one EM step (FP32): E and H read + written once
    per unknown (6 x 2 x 4 B per cell), the voxel byte, the FP32 short-window
    Joule accumulator read + written per node (plus the FP64 fold every 32
    steps: 16 B per node / 32), and the CPML state in the slabs (4 field
    components x (chi high part, chi low part, previous derivative) x
    read + write x 4 B)."""
    cells, nodes = p.n_cells, p.n_nodes
    L = p.cpml_cells
    psi = 0
    n = (p.nx, p.ny, p.nz)
    for a in range(3):
        sides = (p.em_bc[2 * a] == 2) + (p.em_bc[2 * a + 1] == 2)
        if sides:
            area = nodes // (n[a] + 1)
            psi += sides * (L + 1) * area * 4 * 3 * 2 * 4
    return 48 * cells + cells + 8 * nodes + nodes // 2 + psi


def kernel_source_hash(paths):
    """First 16 hex digits of the SHA-256 of the kernel's source files, in order."""
    h = hashlib.sha256()
    for q in paths:
        h.update(open(q, "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_srcs, nx, ny, nz):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (em.cuh and the common.cuh it includes) and on
    this workload (the 1024 x 1024 x 128 package); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
        h = kernel_source_hash(kernel_srcs)
        if t.get("em_step_kernel", {}).get("source_sha256_16") == h and (nx, ny, nz) == (1024, 1024, 128):
            return t["em_step_kernel"]["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def whole_job(ms_local, units_per_step, steps, world, device="cuda"):
    """Each rank times its own replica of the workload; the job's time is the
    slowest rank's (all-reduce MAX when world > 1) and its rate is all ranks'
    units over that time, in G units/s. Returns (ms_total, rate)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        t = torch.tensor([ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_step / (ms / steps * 1e-3) / 1e9


def gpu_arm(args, rank, world):
    import numpy as np
    import torch

    import workloads as W
    from paper_2603_07038_b300 import build as B
    from paper_2603_07038_b300 import cosim as api

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    api.load()
    p = W.layered_package(args.nx, args.ny, seed=2 + rank, nz=args.nz)
    stream = torch.cuda.current_stream()
    total_em = (args.warmup + args.steps + 4) * N_EM
    ctx = api.Context(p, precision=api.COSIM_FP32, stream=stream, use_torch_allocator=True)
    tables = p.source_tables(ctx.dt, total_em)
    ctx.set_sources(tables)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(rec=None):
        ctx.joule(api.COSIM_JOULE_RESET, want_total=False)
        if rec is not None:
            rec[0].record(stream)
        ctx.em_steps(N_EM, accumulate_joule=True)
        if rec is not None:
            rec[1].record(stream)
        ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER, want_total=False)
        ctx.thermal_steps(N_TH)
        if rec is not None:
            rec[2].record(stream)
        ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-30, maxit=N_CG,
                         check_every=N_CG, allow_not_converged=True)
        if rec is not None:
            rec[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    clocks = ClockSampler(("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else (uuid or dev))
    clocks.start()
    time.sleep(0.3)
    l0 = ctx.query(api.COSIM_Q_LAUNCHES)
    t0, t1 = ev(), ev()
    recs = [[ev() for _ in range(4)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0.record(stream)
    for s in range(args.steps):
        step(recs[s])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = int(ctx.query(api.COSIM_Q_LAUNCHES) - l0)
    ms_total = t0.elapsed_time(t1)
    em_ms = sum(r[0].elapsed_time(r[1]) for r in recs)
    th_ms = sum(r[1].elapsed_time(r[2]) for r in recs)
    cg_ms = sum(r[2].elapsed_time(r[3]) for r in recs)
    updates_step = p.n_cells * N_EM + p.n_nodes * N_TH  # EM + thermal; the stress slice's time counts, not its updates
    ms_total, value = whole_job(ms_total, updates_step, args.steps, world)
    ms_step = ms_total / args.steps
    # the paper's own marching (Sec. II-A), outside the timed region: EM steps
    # with sigma(T) and a thermal step at the EM dt after each
    ctx.em_steps(N_CPL, coupled=True)
    c0, c1 = ev(), ev()
    c0.record(stream)
    ctx.em_steps(N_CPL, coupled=True)
    c1.record(stream)
    torch.cuda.synchronize()
    cpl_ms = c0.elapsed_time(c1) / N_CPL
    # the same steps in one launch each (the thermal step inside the EM kernel)
    ctx.em_steps(N_CPL, coupled=True, fused=True)
    c0, c1 = ev(), ev()
    c0.record(stream)
    ctx.em_steps(N_CPL, coupled=True, fused=True)
    c1.record(stream)
    torch.cuda.synchronize()
    cpl_fused_ms = c0.elapsed_time(c1) / N_CPL
    cg = None if args.no_cg_solve else stress_cg_solve(ctx, p, stream)
    em_launch_ms = em_ms / (args.steps * N_EM)
    alg = em_alg_bytes(ctx, p)
    peaks = load_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6400.0
    achieved = alg / (em_launch_ms * 1e-3) / 1e9
    csrc = os.path.join(ROOT, "paper_2603_07038_b300", "csrc")
    traffic = traffic_from_profile([os.path.join(csrc, "em.cuh"), os.path.join(csrc, "common.cuh")], args.nx, args.ny, args.nz)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded layered package generator)",
        "config": {"workload": workload_name(args.nx, args.ny, args.nz), "nx": args.nx, "ny": args.ny, "nz": args.nz, "cells": p.n_cells,
                   "nodes": p.n_nodes, "step": f"{N_EM} EM steps + Joule + {N_TH} thermal steps + "
                                           f"stress slice ({N_CG} PCG iterations); value counts the EM cell-steps "
                                           f"and thermal node-steps over the whole step's time",
                   "signal_lines": len(p.sources), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (state ~%.0f GB resident)" % (ctx.query(api.COSIM_Q_BYTES_RESIDENT) / 1e9)},
        "phases": {"em_thermal_gcell_updates_s": round(updates_step * args.steps / ((em_ms + th_ms) * 1e-3) / 1e9, 3),
                   "em_gcell_steps_s": round(p.n_cells * N_EM * args.steps / (em_ms * 1e-3) / 1e9, 3),
                   "em_ms_per_step": round(em_launch_ms, 4),
                   "thermal_gnode_steps_s": round(p.n_nodes * N_TH * args.steps / (th_ms * 1e-3) / 1e9, 3),
                   "stress_slice_ms": round(cg_ms / args.steps, 3),
                   "coupled_ms_per_step": round(cpl_ms, 4),
                   "coupled_gcell_steps_s": round(p.n_cells / (cpl_ms * 1e-3) / 1e9, 3),
                   "coupled_one_launch_ms_per_step": round(cpl_fused_ms, 4),
                   "stress_cg_s_per_solve": cg["s_per_solve"] if cg else None},
        "stress_cg": cg,
        "roofline": {"kernel": "em_step_kernel", "bound": "hbm", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "alg_bytes_per_launch": alg,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback 6.4 TB/s"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_arm(args, p, stream, world)
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args, p)
    ctx.close()
    if rank == 0 and not args.no_batch:
        out["batched"] = batched_arm(args)
    if rank == 0 and not args.no_serve:
        out["serving"] = serving_arm(args)
    return out


def stress_cg_solve(ctx, p, stream, rise=60.0, rtol=1e-9, maxit=20000):
    """One whole stress solve (after the timed region) at the accuracy the
    displacement and stress results need: FP32 Jacobi-PCG (FP64 dot products)
    inside FP64 iterative refinement, to a 1e-9 relative residual of the FP64
    system (each inner solve to 1e-4), bottom face clamped, under
    a synthetic hot spot (a Gaussian rise of `rise` K centred on the package,
    width sqrt(0.05) of each lateral extent, falling linearly from the top to
    a fifth of it at the bottom) built on the device and written through the
    C ABI. The EM burst of a bench step heats the package by nano-kelvins
    only, so that load would not exercise the solver's convergence."""
    import torch

    from paper_2603_07038_b300 import cosim as api
    f64 = dict(dtype=torch.float64, device="cuda")
    gx = torch.exp(-((torch.arange(p.nx + 1, **f64) / p.nx - 0.5) ** 2) / 0.05)
    gy = torch.exp(-((torch.arange(p.ny + 1, **f64) / p.ny - 0.5) ** 2) / 0.05)
    gz = torch.linspace(0.2, 1.0, p.nz + 1, **f64)
    T = 300.0 + rise * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    ctx.write(api.COSIM_F_T, T.reshape(-1))
    del T
    torch.cuda.empty_cache()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=rtol, maxit=maxit, check_every=64,
                           allow_not_converged=True, refine=True, inner_rtol=1e-4)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    return {"s_per_solve": round(sec, 3), "iters": int(rep["iters"]), "refine_steps": int(rep["refine_steps"]),
            "relres_fp64": float(rep["relres"]), "rtol": rtol,
            "converged": rep["status"] == api.COSIM_OK, "ms_per_iter": round(sec * 1e3 / max(rep["iters"], 1), 3),
            "dofs": 3 * p.n_nodes,
            "precision": "FP32 Jacobi-PCG (FP64 dots) in FP64 iterative refinement; relres_fp64 is the true "
                         "residual ||f - K u|| / ||f|| of the FP64 system",
            "load": "synthetic %.0f K hot spot, bottom clamped" % rise}


def batched_arm(args, n=64, win=32, windows=3, seed=4, streams=4):
    """The batched-design workload (after the timed region): n seeded package
    designs, grids drawn uniformly from 128^3, 256^2 x 64, 384^2 x 64 and
    512^2 x 96 cells, TSV pitch 4-8 voxels, per-design port lines and PRBS
    bursts, FP32 fields with FP64 Joule totals, each advanced `windows`
    32-step windows of EM steps with Joule accumulation, in four forms:
      sequential: one design at a time, each replaying its own captured graph;
      batch: one launch per step over every design's tiles (captured graph);
      batch_persistent: the same with a persistent launch taking the tiles
        from a device counter, largest designs first (captured graph);
      streams: the designs spread over `streams` CUDA streams, each replaying
        its own graph (the serving loop's form).
    Rates are cell-steps of all designs per second; the projection to the
    2 ns burst (314,701 steps per design at this dt) gives designs/hour of
    EM bursts. One warm-up window per form."""
    import torch

    import workloads as W
    from paper_2603_07038_b300 import cosim as api
    from paper_2603_07038_b300 import serving as S
    specs = S.design_mix(n, seed=seed, em_steps=win * windows)
    probs = [W.layered_package(sp.nx, sp.ny, seed=100 + sp.seed, nz=sp.nz, tsv_pitch=sp.tsv_pitch, n_lines=8)
             for sp in specs]
    cells = sum(p.n_cells for p in probs)
    total = 4 * (windows + 1) * win
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {"designs": n, "cells_total": cells, "steps_timed": windows * win,
           "grids": {f"{a}x{b}x{c}": sum(1 for sp in specs if (sp.nx, sp.ny, sp.nz) == (a, b, c))
                     for a, b, c in S.DESIGN_GRIDS}}

    def make(stream_of):
        ctxs = []
        for d, (sp, p) in enumerate(zip(specs, probs)):
            c = api.Context(p, precision=api.COSIM_FP32, stream=stream_of(d), use_torch_allocator=True)
            c.set_sources(p.source_tables(c.dt, total, sp.t0))
            c.joule(api.COSIM_JOULE_RESET, want_total=False)
            ctxs.append(c)
        return ctxs

    def timed(run, sync_streams):
        run(1)  # warm-up window
        torch.cuda.synchronize()
        t0, t1 = ev(), ev()
        base = sync_streams[0]
        t0.record(base)
        for st in sync_streams[1:]:
            st.wait_event(t0)
        run(windows)
        for st in sync_streams[1:]:
            e = ev()
            e.record(st)
            base.wait_event(e)
        t1.record(base)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) * 1e-3

    rates = {}
    s0 = torch.cuda.Stream()
    ctxs = make(lambda d: s0)
    for c in ctxs:
        c.em_graph_capture(win)
    sec = timed(lambda w: [c.em_graph_launch(w) for c in ctxs], [s0])
    rates["sequential"] = cells * windows * win / sec / 1e9
    for name, pers in (("batch", False), ("batch_persistent", True)):
        b = api.Batch(ctxs, persistent=pers)
        b.graph_capture(win)
        sec = timed(lambda w, b=b: b.graph_launch(w), [s0])
        rates[name] = cells * windows * win / sec / 1e9
        b.close()
    dt = ctxs[0].dt
    for c in ctxs:
        c.close()
    del ctxs
    torch.cuda.empty_cache()
    sts = [torch.cuda.Stream() for _ in range(streams)]
    ctxs = make(lambda d: sts[d % streams])
    for c in ctxs:
        c.em_graph_capture(win)
    sec = timed(lambda w: [c.em_graph_launch(w) for c in ctxs], sts)
    rates["streams"] = cells * windows * win / sec / 1e9
    for c in ctxs:
        c.close()
    del ctxs
    torch.cuda.empty_cache()
    burst = int(round(2e-9 / dt))
    out["gcell_steps_s"] = {k: round(v, 3) for k, v in rates.items()}
    out["em_burst_designs_per_hour"] = {k: round(3600.0 * v * 1e9 / (cells / n * burst), 1) for k, v in rates.items()}
    out["note"] = ("designs/hour of 2 ns EM bursts (%d steps per design) projected from the timed windows; "
                   "the batch forms are one launch per step for all %d designs" % (burst, n))
    return out


def serving_arm(args, workers=4, config5=False):
    """Continuous batching of a seeded design trace (after the timed region).
    Burst-length-scaled variant: designs from the batched mix at half lateral
    size (config5: at full size, with 10 % of the requests the full-scale
    1024 x 1024 x 128 package), args.serve_em_steps EM steps (graph-replayed),
    2000 thermal steps and a converged stress solve (1e-6) per request;
    Poisson arrivals at 80 % of the capacity measured on the first designs run
    back to back. Latencies include queueing."""
    from paper_2603_07038_b300 import serving as S
    if config5:
        specs = S.design_mix(args.serve_n, seed=12, em_steps=args.serve_em_steps, thermal_steps=2000,
                             big_fraction=0.1)
    else:
        specs = S.design_mix(args.serve_n, seed=11, em_steps=args.serve_em_steps, thermal_steps=2000, scale=0.5)
    specs = [dataclasses.replace(s, cg_maxit=100000) for s in specs]
    runner = S.DesignRunner(specs, workers=workers)
    runner.run(specs[0], 0)  # warm-up: module load, allocator pools
    t = time.perf_counter()
    calib = specs[:min(4, len(specs))]
    for s in calib:
        runner.run(s, 0)
    per_design = (time.perf_counter() - t) / len(calib)
    rate = 0.8 / per_design
    arr = S.poisson_arrivals(len(specs), rate, seed=11)
    rep = S.serve(specs, arr, runner.run, workers=workers, footprint=S.footprint_bytes)
    # the served form as a closed batch (everything queued at t = 0), the
    # like-for-like comparison with the plain form below
    rep_batch = S.serve(specs, [0.0] * len(specs), runner.run, workers=workers, footprint=S.footprint_bytes)
    # the plain form on the same GPU: one design at a time, step-by-step
    # launches, the same (autotuned) launch shapes, everything queued at t = 0
    plain = S.DesignRunner(specs, workers=1, use_graph=False, autotune=True)
    plain.run(specs[0], 0)
    rep_plain = S.serve(specs, [0.0] * len(specs), plain.run, workers=1, footprint=S.footprint_bytes)
    # same shapes, deterministic kernels, graph replays equal to plain steps:
    # every figure of every design is identical in the three runs
    keys = ("joule_J", "T_max", "vm_max", "cg_iters", "cg_relres")
    same = all(all(r["records"][q].result[k] == rep_plain["records"][q].result[k] for k in keys)
               for r in (rep, rep_batch) for q in range(len(specs)))
    conv = all(r.result["cg_relres"] <= specs[r.job].cg_rtol for r in rep["records"])
    cells = sum(s.cells for s in specs)
    return {"variant": "burst-length-scaled (%d EM steps per request, not the 2 ns burst), ~80%% offered load"
                       % specs[0].em_steps,
            "mix": "config-5 mix: full-size design grids, %d of %d requests 1024x1024x128" % (
                sum(1 for sp in specs if (sp.nx, sp.ny, sp.nz) == S.FULL_GRID), len(specs))
                   if config5 else "design grids at half lateral size",
            "requests": len(specs), "workers": workers, "arrival_rate_per_s": round(rate, 3),
            "p50_s": round(rep["p50_s"], 4), "p99_s": round(rep["p99_s"], 4),
            "designs_per_hour": round(rep["designs_per_hour"], 1), "makespan_s": round(rep["makespan_s"], 3),
            "batch_designs_per_hour": round(rep_batch["designs_per_hour"], 1),
            "plain_designs_per_hour": round(rep_plain["designs_per_hour"], 1),
            "plain_note": "same requests one at a time, no graphs, the same launch shapes, all queued at t=0",
            "results_identical": bool(same), "cg_converged": bool(conv),
            "per_request": "%d EM steps, %d thermal steps, stress solve to rtol %g" % (
                specs[0].em_steps, specs[0].thermal_steps, specs[0].cg_rtol),
            "mean_cells": int(cells / len(specs)), "em_path": "captured CUDA graph, 32-step windows"}


def e2e_arm(args, p, stream, world, nsteps=2):
    """Same step through the public C ABI with host buffers: every step
    uploads the package from pinned host memory (cosim_create copies voxels,
    spacings, materials; cosim_set_sources the ports), runs the pass and reads
    the temperature (started as soon as it is final, while the stress solve
    runs) and von Mises fields back into pinned host memory."""
    import numpy as np
    import torch

    from paper_2603_07038_b300 import cosim as api
    mat_pinned = torch.empty(p.mat.shape, dtype=torch.uint8).pin_memory()
    mat_pinned.numpy()[...] = p.mat
    p.mat = mat_pinned.numpy()
    T_host = torch.empty(p.n_nodes, dtype=torch.float32).pin_memory().numpy()
    VM_host = torch.empty(p.n_cells, dtype=torch.float32).pin_memory().numpy()
    times = []
    h2d = d2h = 0
    for s in range(nsteps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx = api.Context(p, precision=api.COSIM_FP32, stream=stream, use_torch_allocator=True)
        tables = p.source_tables(ctx.dt, N_EM)
        ctx.set_sources(tables)
        ctx.em_steps(N_EM, True)
        ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER, want_total=False)
        ctx.thermal_steps(N_TH)
        # the temperature is final here: its copy to the host overlaps the solve
        api.cosim_read_fields_async(ctx.h, api.COSIM_F_T, T_host)
        ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=1e-30, maxit=N_CG,
                         check_every=N_CG, allow_not_converged=True)
        api.cosim_read_fields(ctx.h, api.COSIM_F_VM, VM_host)
        api.cosim_wait_reads(ctx.h)
        ctx.close()
        torch.cuda.synchronize()
        if s > 0:  # the first pass warms the caching allocator
            times.append(time.perf_counter() - t)
        h2d = (p.mat.nbytes + 8 * (p.nx + p.ny + p.nz) + 80 * len(p.materials)
               + sum(e.nbytes + a.nbytes for _, e, a in tables))
        d2h = T_host.nbytes + VM_host.nbytes
    sec = statistics.median(times)
    upd = p.n_cells * N_EM + p.n_nodes * N_TH
    return {"value": round(upd / sec / 1e9, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "seconds_per_step": round(sec, 3),
            "note": "cosim_create + set_sources + pass + T (cosim_read_fields_async, overlapping the stress solve) "
                    "and VM (cosim_read_fields) to pinned host, per step"}


# ---------------------------------------------------------------- oracle (CPU) arm

def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_point_seconds(job):
    """Per-point seconds of the FP64 oracle on one package window (a crop of
    all 128 layers, CPML faces included): (EM cell-step, thermal node-step,
    HEX8 matvec node). Runs in a worker process of OracleBaseline."""
    wp, n_em, n_th, n_mv = job
    import numpy as np

    import oracle
    from workloads import constraints as BC
    o = oracle.OracleSim(wp)
    rng = np.random.default_rng(0)
    for a in range(3):
        o.E[a][:] = rng.standard_normal(o.g.n_nodes) * 1e-3
    t = time.perf_counter()
    o.em_steps(n_em)
    t_em = (time.perf_counter() - t) / (n_em * wp.n_cells)
    o.P = rng.random(o.g.n_nodes) * 1e-9
    t = time.perf_counter()
    o.thermal_steps(n_th)
    t_th = (time.perf_counter() - t) / (n_th * wp.n_nodes)
    fixed = BC.clamped_bottom(wp)
    u = rng.standard_normal(3 * wp.n_nodes) * 1e-9
    t = time.perf_counter()
    for _ in range(n_mv):
        o.matvec(fixed, u)
    t_mv = (time.perf_counter() - t) / (n_mv * wp.n_nodes)
    return t_em, t_th, t_mv


class OracleBaseline:
    """The FP64 CPU oracle, as it stands, on the host cores: one worker process
    per core (spawned: safe after CUDA initialisation), each running the
    oracle on its own window of the package. A sample times n_em EM steps,
    n_th thermal steps and n_mv HEX8 matvecs per window and scales the
    per-point times to the full step (a CG iteration counted as its matvec);
    the all-cores rate is the sum of the workers' rates measured while all
    run at once, the single-thread rate one worker running alone."""

    def __init__(self, p_full, win=(64, 64), procs=None):
        import dataclasses as dc
        import multiprocessing as mp

        import oracle
        import workloads as W
        oracle.build()
        self.p = p_full
        self.win = win
        self.procs = procs or host_cores()
        nwx, nwy = p_full.nx // win[0], p_full.ny // win[1]
        self.windows = []
        for q in range(self.procs):  # windows spread over the package, CPML corners included
            x0, y0 = (q % nwx) * win[0], ((q // nwx) % nwy) * win[1]
            wp = W.crop(p_full, (x0, y0, 0), (x0 + win[0], y0 + win[1], p_full.nz))
            self.windows.append(dc.replace(wp, sources=[]))
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def _rate(self, t):
        t_em, t_th, t_mv = t
        p = self.p
        sec = N_EM * p.n_cells * t_em + N_TH * p.n_nodes * t_th + N_CG * p.n_nodes * t_mv
        return (p.n_cells * N_EM + p.n_nodes * N_TH) / sec / 1e9

    def sample(self, n_em=2, n_th=2, n_mv=1):
        """all cores: (G updates/s, wall seconds of the sample)"""
        t = time.perf_counter()
        res = self.pool.map(_oracle_point_seconds, [(w, n_em, n_th, n_mv) for w in self.windows], chunksize=1)
        return sum(self._rate(r) for r in res), time.perf_counter() - t

    def single(self, n_em=2, n_th=2, n_mv=1):
        """one worker alone: G updates/s"""
        return self._rate(self.pool.apply(_oracle_point_seconds, ((self.windows[0], n_em, n_th, n_mv),)))

    def describe(self, n_em, n_th, n_mv, samples):
        return (f"FP64 oracle, {self.procs} worker processes on {self.procs} host cores ({cpu_model()}), each on its "
                f"own {self.win[0]}x{self.win[1]}x{self.p.nz} window of the package: {n_em} EM steps, {n_th} thermal "
                f"steps, {n_mv} HEX8 matvec per window and sample, median of {samples} samples, scaled per grid point "
                f"to the full step (a CG iteration counted as its matvec)")


# one sample of the baseline: per window, about 3 s of oracle work
CPU_SAMPLE = dict(n_em=6, n_th=6, n_mv=2)


def cpu_baseline(args, p, samples=6):
    ob = OracleBaseline(p)
    try:
        ob.sample(1, 1, 1)  # worker start-up and first-touch, untimed
        vals = [ob.sample(**CPU_SAMPLE)[0] for _ in range(samples)]
        single = statistics.median([ob.single(**CPU_SAMPLE) for _ in range(2)])
    finally:
        ob.close()
    return {"value": round(statistics.median(vals), 6), "unit": UNIT, "cores": ob.procs, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": host_cores(),
            "sample": ob.describe(samples=samples, **CPU_SAMPLE),
            "spread": round((max(vals) - min(vals)) / statistics.median(vals), 4),
            "single_thread": {"value": round(single, 6), "cores": 1}}


def reference_arm(args):
    import workloads as W
    p = W.layered_package(args.nx, args.ny, seed=2, nz=args.nz)
    ob = OracleBaseline(p)
    try:
        for _ in range(args.warmup):
            ob.sample(**CPU_SAMPLE)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(ob.sample(**CPU_SAMPLE)[0])
        wall = time.perf_counter() - t0
    finally:
        ob.close()
    v = statistics.median(vals)
    upd = p.n_cells * N_EM + p.n_nodes * N_TH
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / max(args.steps, 1) * 1e3, 1),
            "full_step_ms_extrapolated": round(upd / (v * 1e9) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded layered package generator)",
            "config": {"workload": workload_name(args.nx, args.ny, args.nz), "nx": args.nx, "ny": args.ny, "nz": args.nz,
                       "step": f"a bounded sample of the step ({N_EM} EM steps + {N_TH} thermal steps + {N_CG} CG "
                               f"iterations on the package) on windows of it, as cpu_baseline.sample describes; "
                               f"ms_per_step is the sample's wall time, value its per-point rate, "
                               f"full_step_ms_extrapolated the whole package's step at that rate"},
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": ob.procs, "kind": "oracle",
                             "cpu_model": cpu_model(), "nproc": host_cores(),
                             "sample": ob.describe(samples=args.steps, **CPU_SAMPLE), "wall_s": round(wall, 1),
                             "spread": round((max(vals) - min(vals)) / v, 4)},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)))
        return
    if args.serve_config5:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2603_07038_b300 import build as B
        B.build()
        print(json.dumps({"serving_config5": serving_arm(args, config5=True)}))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = gpu_arm(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
