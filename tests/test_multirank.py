"""The benchmark's multi-GPU form is independent replicas (one per rank, no
data-path collective): a barrier brackets the timed region and the job's
time is the slowest rank's. Checked here with world_size 2 on CPU (gloo)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.whole_job(100.0 + 50.0 * rank, 2e9, 4, world, device="cpu")
    torch.distributed.barrier()
    q.put((rank, ms, rate))
    torch.distributed.destroy_process_group()


def test_whole_job_time_is_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 150.0  # the slower rank's 150 ms for 4 steps
        assert rate == pytest.approx(2 * 2e9 / (150.0 / 4 * 1e-3) / 1e9)  # both replicas' work


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.whole_job(80.0, 1e9, 2, 1)
    assert ms == 80.0 and rate == pytest.approx(1e9 / 0.04 / 1e9)


def test_reference_arm_prints_only_on_rank_zero():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
