"""Batched execution and a continuous serving loop over many package designs
on one GPU.

A design (one request) runs the whole hot path end to end through the C-ABI:
EM burst with Joule accumulation (replayed from a captured CUDA graph in
32-step windows), the burst-averaged Joule source, explicit thermal steps,
the clamped-bottom thermoelastic solve and von Mises stress (Sec. II-A,
II-B). Several designs run at once, each on its own CUDA stream from a
worker thread (the C-ABI releases the GIL while it launches); admission keeps
the summed device footprint of the running designs under an HBM budget.
Contexts share no device state and every kernel is deterministic, so a
design's results do not depend on what runs beside it.

The scheduler (`serve`) is independent of the GPU work: it takes any
``run(job, worker) -> dict`` callable, which the tests replace with a fake.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from typing import Callable, Sequence

import numpy as np

# Grid sizes of the batched design mix (cells): 128^3, 256^2 x 64,
# 384^2 x 64, 512^2 x 96.
DESIGN_GRIDS = ((128, 128, 128), (256, 256, 64), (384, 384, 64), (512, 512, 96))


@dataclasses.dataclass(frozen=True)
class DesignSpec:
    """One design request. em_steps is rounded up to whole 32-step windows."""
    seed: int
    nx: int
    ny: int
    nz: int
    tsv_pitch: int = 5
    em_steps: int = 256
    thermal_steps: int = 100
    cg_rtol: float = 1e-6
    cg_maxit: int = 500
    # start of the simulated EM window: a short (scaled) burst samples the
    # port waveforms around the first bit edge instead of the quiet lead-in
    t0: float = 50e-12

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


# the full-scale package grid that the serving trace mixes in
FULL_GRID = (1024, 1024, 128)


def design_mix(n: int, seed: int = 0, em_steps: int = 256, thermal_steps: int = 100, scale: float = 1.0,
               grids: Sequence = DESIGN_GRIDS, big_fraction: float = 0.0) -> list[DesignSpec]:
    """n seeded designs: grid drawn uniformly from ``grids`` (lateral size
    multiplied by ``scale``), TSV pitch uniform in 4..8 voxels (40-80 um);
    with probability ``big_fraction`` a request is the full-scale
    1024 x 1024 x 128 package instead (not scaled)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n):
        big = big_fraction > 0 and rng.random() < big_fraction
        nx, ny, nz = grids[int(rng.integers(0, len(grids)))]
        if big:
            out.append(DesignSpec(seed=s, nx=FULL_GRID[0], ny=FULL_GRID[1], nz=FULL_GRID[2],
                                  tsv_pitch=int(rng.integers(4, 9)), em_steps=em_steps, thermal_steps=thermal_steps))
            continue
        nx, ny = max(48, int(round(nx * scale))), max(48, int(round(ny * scale)))
        out.append(DesignSpec(seed=s, nx=nx, ny=ny, nz=nz, tsv_pitch=int(rng.integers(4, 9)),
                              em_steps=em_steps, thermal_steps=thermal_steps))
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a seeded Poisson process; the first arrives at 0."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n)
    gaps[0] = 0.0
    return np.cumsum(gaps)


def footprint_bytes(spec: DesignSpec, elem_bytes: int = 4) -> int:
    """Upper estimate of a design's resident device bytes (context state:
    double-buffered E/H, Joule totals, temperature, mechanics vectors, CPML
    slabs), used for admission; tests check it bounds the measured figure."""
    px = (spec.nx + 1 + 31) // 32 * 32
    npad = px * (spec.ny + 1) * (spec.nz + 1)
    return int(npad * (52 * elem_bytes + 24) + 6 * spec.cells + (64 << 20))


def percentile(x, q) -> float:
    """q-th percentile (0..100) with linear interpolation between order statistics."""
    return float(np.percentile(np.asarray(x, np.float64), q)) if len(x) else float("nan")


@dataclasses.dataclass
class Record:
    job: int
    arrival: float
    start: float = float("nan")
    finish: float = float("nan")
    worker: int = -1
    result: dict | None = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def serve(jobs: Sequence, arrivals: Sequence[float], run: Callable, workers: int = 4,
          budget_bytes: float = 150e9, footprint: Callable = lambda job: 0, clock=time.perf_counter) -> dict:
    """Continuous batching: whenever a worker is free, start the earliest
    arrived job that has not started, provided the running jobs' footprints
    plus its own stay within ``budget_bytes`` (jobs start in arrival order; a
    job larger than the whole budget runs alone). Latency is measured from
    arrival to completion (queueing included). Returns p50/p99 latency,
    designs per hour over the makespan, and the per-job records."""
    n = len(jobs)
    recs = [Record(job=q, arrival=float(arrivals[q])) for q in range(n)]
    order = sorted(range(n), key=lambda q: (recs[q].arrival, q))
    lock = threading.Condition()
    state = {"next": 0, "used": 0.0, "running": 0, "error": None}
    t0 = clock()

    def now():
        return clock() - t0

    def take(w):
        with lock:
            while True:
                if state["error"] is not None or state["next"] >= n:
                    return None
                q = order[state["next"]]
                wait = recs[q].arrival - now()
                need = float(footprint(jobs[q]))
                fits = state["used"] + need <= budget_bytes or state["running"] == 0
                if wait <= 0 and fits:
                    state["next"] += 1
                    state["used"] += need
                    state["running"] += 1
                    recs[q].start, recs[q].worker = now(), w
                    return q, need
                lock.wait(timeout=max(wait, 0.0) if wait > 0 else 0.05)

    def worker(w):
        while True:
            got = take(w)
            if got is None:
                return
            q, need = got
            try:
                res = run(jobs[q], w)
            except BaseException as e:  # surface the first failure, stop the others
                with lock:
                    state["error"] = e
                    state["running"] -= 1
                    state["used"] -= need
                    lock.notify_all()
                return
            with lock:
                recs[q].finish, recs[q].result = now(), res
                state["used"] -= need
                state["running"] -= 1
                lock.notify_all()

    threads = [threading.Thread(target=worker, args=(w,), daemon=True) for w in range(workers)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if state["error"] is not None:
        raise state["error"]
    lat = [r.latency for r in recs]
    makespan = max(r.finish for r in recs) if recs else 0.0
    return {"n": n, "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "designs_per_hour": 3600.0 * n / makespan if makespan > 0 else float("nan"),
            "makespan_s": makespan, "records": recs}


class DesignRunner:
    """Runs a DesignSpec on the GPU: one CUDA stream per worker, packages
    generated up front (request payloads), the context created, used and
    destroyed inside the job. ``run(spec, worker)`` returns summary figures and
    the timed phases; ``keep_fields`` also returns T, u and von Mises."""

    def __init__(self, specs: Sequence[DesignSpec], workers: int, precision=None, keep_fields=False,
                 use_graph=True, autotune=True):
        import torch

        import workloads as W
        from . import cosim as api
        self.api, self.torch = api, torch
        self.precision = api.COSIM_FP32 if precision is None else precision
        self.keep = keep_fields
        self.use_graph = use_graph
        self.problems = {s: W.layered_package(s.nx, s.ny, seed=s.seed, nz=s.nz, tsv_pitch=s.tsv_pitch, n_lines=8)
                         for s in specs}
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self.autotune = autotune
        if autotune:  # tune each grid shape once, before any request runs
            for shape in {(s.nx, s.ny, s.nz): s for s in specs}.values():
                c = api.Context(self.problems[shape], precision=self.precision, stream=self.streams[0],
                                use_torch_allocator=True)
                c.autotune()
                c.close()

    def run(self, spec: DesignSpec, worker: int) -> dict:
        api = self.api
        p = self.problems[spec]
        stream = self.streams[worker]
        win = 32
        n_em = (spec.em_steps + win - 1) // win * win
        t = [time.perf_counter()]
        # the caching allocator: a plain cudaFree would synchronise the whole
        # device and stall the designs running beside this one
        ctx = api.Context(p, precision=self.precision, stream=stream, use_torch_allocator=True)
        try:
            if self.autotune:
                ctx.autotune()  # the shape's cached choice
            ctx.set_sources(p.source_tables(ctx.dt, n_em, spec.t0))
            ctx.joule(api.COSIM_JOULE_RESET, want_total=False)
            if self.use_graph:
                ctx.em_graph_capture(win)
                ctx.em_graph_launch(n_em // win)
            else:
                ctx.em_steps(n_em)
            energy = ctx.joule(api.COSIM_JOULE_FINALIZE_AVG_POWER)
            t.append(time.perf_counter())
            ctx.thermal_steps(spec.thermal_steps)
            rep = ctx.stress_solve(bc=api.COSIM_MECH_CLAMPED_BOTTOM, T_ref=300.0, rtol=spec.cg_rtol,
                                   maxit=spec.cg_maxit, allow_not_converged=True)
            T = ctx.read(api.COSIM_F_T, np.float32)
            vm = ctx.read(api.COSIM_F_VM, np.float32)
            t.append(time.perf_counter())
            out = {"cells": spec.cells, "em_steps": n_em, "joule_J": energy, "T_max": float(T.max()),
                   "vm_max": float(vm.max()), "cg_iters": int(rep["iters"]), "cg_relres": float(rep["relres"]),
                   "bytes": int(ctx.query(api.COSIM_Q_BYTES_RESIDENT)),
                   "em_s": t[1] - t[0], "rest_s": t[2] - t[1]}
            if self.keep:
                out["T"] = T
                out["vm"] = vm
                out["u"] = np.stack([ctx.read(api.COSIM_F_UX + c, np.float32) for c in range(3)])
            return out
        finally:
            ctx.close()
