"""Host logic of the serving loop (no GPU): design mix, arrivals, admission
under an HBM budget, arrival-order starts, latency percentiles."""
import threading
import time

import numpy as np
import pytest

from paper_2603_07038_b300 import serving as S


def test_design_mix_is_seeded_and_uses_the_grid_set():
    a = S.design_mix(64, seed=3)
    b = S.design_mix(64, seed=3)
    assert a == b
    assert {(d.nx, d.ny, d.nz) for d in a} <= set(S.DESIGN_GRIDS)
    assert len({(d.nx, d.ny, d.nz) for d in a}) == len(S.DESIGN_GRIDS)  # 64 draws hit all four
    assert all(4 <= d.tsv_pitch <= 8 for d in a)
    half = S.design_mix(8, seed=3, scale=0.5)
    assert all(d.nx == max(48, g[0] // 2) for d, g in zip(half, [(x.nx, x.ny) for x in S.design_mix(8, seed=3)]))


def test_poisson_arrivals():
    t = S.poisson_arrivals(20000, rate_per_s=4.0, seed=1)
    assert t[0] == 0 and np.all(np.diff(t) >= 0)
    assert abs(np.mean(np.diff(t)) - 0.25) < 0.01  # mean gap 1/rate
    assert np.array_equal(t, S.poisson_arrivals(20000, 4.0, seed=1))


def test_percentile_matches_definition():
    x = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert S.percentile(x, 50) == 3.0
    assert S.percentile(x, 100) == 5.0
    assert abs(S.percentile(list(range(101)), 99) - 99.0) < 1e-12


def test_serve_respects_budget_and_arrival_order():
    jobs = list(range(12))
    arrivals = [0.0, 0.0, 0.0, 0.01, 0.01, 0.02, 0.02, 0.03, 0.2, 0.2, 0.21, 0.3]
    size = {q: (3 if q % 3 == 0 else 1) for q in jobs}
    lock = threading.Lock()
    live = {"used": 0, "peak": 0, "running": 0, "max_running": 0}

    def run(job, worker):
        with lock:
            live["used"] += size[job]
            live["running"] += 1
            live["peak"] = max(live["peak"], live["used"])
            live["max_running"] = max(live["max_running"], live["running"])
        time.sleep(0.02)
        with lock:
            live["used"] -= size[job]
            live["running"] -= 1
        return {"job": job, "worker": worker}

    rep = S.serve(jobs, arrivals, run, workers=3, budget_bytes=4, footprint=lambda q: size[q])
    recs = rep["records"]
    assert live["peak"] <= 4 and live["max_running"] <= 3
    assert all(r.result["job"] == r.job for r in recs)
    assert all(r.start >= r.arrival - 1e-9 and r.finish > r.start for r in recs)
    starts = [r.start for r in sorted(recs, key=lambda r: (r.arrival, r.job))]
    assert starts == sorted(starts)  # jobs start in arrival order
    lat = [r.latency for r in recs]
    assert rep["p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert rep["p99_s"] == pytest.approx(np.percentile(lat, 99))
    assert rep["designs_per_hour"] == pytest.approx(3600 * 12 / rep["makespan_s"])


def test_oversized_job_runs_alone_and_errors_propagate():
    rep = S.serve([0, 1], [0.0, 0.0], lambda j, w: {}, workers=2, budget_bytes=1, footprint=lambda j: 5)
    assert rep["n"] == 2

    def boom(j, w):
        raise RuntimeError("job failed")
    with pytest.raises(RuntimeError):
        S.serve([0, 1, 2], [0, 0, 0], boom, workers=2)


def test_footprint_estimate_grows_with_the_grid():
    small = S.DesignSpec(seed=0, nx=128, ny=128, nz=128)
    big = S.DesignSpec(seed=0, nx=512, ny=512, nz=96)
    assert S.footprint_bytes(big) > 4 * S.footprint_bytes(small) > 0
