"""Host-side logic of bench.py: rank reduction and whole-job rate (CPU, gloo,
world size 2), and the reference arm's rank handling."""
from __future__ import annotations

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 10 ms: the job's time is the slowest rank's
        ms = bench.max_over_ranks(10.0 * (rank + 1), world, device="cpu")
        rate = bench.whole_job_rate(1000.0, world, ms)
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "cpu_tents": 1})(),
                                  rank, world) if rank == 1 else "skip"
        out.put((rank, ms, rate, ref))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, ref in res:
        assert ms == 20.0
        assert rate == pytest.approx(1000.0 * 2 / 0.020)
        if rank == 1:
            assert ref is None       # only rank 0 runs and prints the reference arm


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(505400, 1, 42.0) == pytest.approx(505400 / 0.042)


def test_cpu_baseline_runs_single_threaded_blas():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        assert os.environ[v] == "1"
