"""The multi-process side of bench.py on CPU: two gloo ranks (127.0.0.1) reduce
their step times to the slowest one and report the whole job's rate, as the
bench does for one replica per GPU (the render path has no exchange step)."""
from __future__ import annotations

import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = bench.env_rank()
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        t_max = bench.max_over_ranks(ms, dist, device="cpu")
        rate = bench.whole_job_rate(1024 * 5, w, t_max / 1e3)
        out.put((r, local, w, t_max, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_the_slowest_and_report_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1] and all(g[2] == 2 for g in got)
    for _, _, _, t_max, rate in got:
        assert t_max == pytest.approx(150.0)
        assert rate == pytest.approx(1024 * 5 * 2 / 0.150)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
