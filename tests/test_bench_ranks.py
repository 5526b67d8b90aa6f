"""The multi-rank path of bench.py on CPU (gloo, world size 2): the step time
is the maximum over the ranks and the throughput counts the products of
every replica."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 1000, world, "cpu")
    dist.barrier()
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 15.0                                  # the slower rank
        assert abs(value - 2 * 1000 / 0.015) < 1e-6        # both replicas' products


def test_single_rank_needs_no_collective():
    import bench
    assert bench.aggregate_over_ranks(20.0, 500, 1, "cpu") == (20.0, 500 / 0.02)
