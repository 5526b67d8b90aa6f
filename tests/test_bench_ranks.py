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


def test_roofline_work_counts_match_their_definitions():
    """bench.py's multiply counts at N = 8192, L = 4 (K = 15): per product
    10KN + 3K (N/2) log N 3 + 3N (3K + 2KL + 6L + 2) = 13.11 M, the
    formulation the kernel runs (an earlier one needed 6K + 2KL + 9L per
    rounded coefficient: 14.46 M, kept only as a note); per entry L (L+2)
    forward NTTs of 10 per butterfly plus 7N, 2 L^2 N 10 key products,
    2 L N 7 final reductions = 17.24 M; the grouped mode counts the tensor
    per product and the rest per group; the bench line's fraction is that
    work over the kernel's time over 152 x 64 x 2070 MHz."""
    import bench
    N, L, K = 8192, 4, 15
    assert bench.tensor_base_size(13, 4) == K
    per_product = 10 * K * N + 3 * K * (N // 2) * 13 * 3 + 3 * N * (3 * K + 2 * K * L + 6 * L + 2)
    assert bench.mults_per_product(N, L) == per_product == 13_111_296
    assert bench.mults_per_product_retired(N, L) == 14_462_976
    assert bench.mults_per_entry(N, L) == L * (L + 2) * ((N // 2) * 13 * 10 + 7 * N) + 2 * L * L * N * 10 + 2 * L * N * 7
    assert abs(bench.mults_per_entry(N, L) / 1e6 - 17.24) < 0.01
    assert bench.mults(10, 2, N, L) == 10 * per_product + 2 * bench.mults_per_entry(N, L)
    assert bench.mults(10, 2, N, L, groups=1) == 10 * 10 * K * N + (per_product - 10 * K * N) + 2 * bench.mults_per_entry(N, L)
    # the headline launch: 130,240 products over 4,096 entries
    rl = bench.alu_roofline(130_240, 4_096, N, L, 262.9)
    work = 130_240 * per_product + 4_096 * bench.mults_per_entry(N, L)
    assert rl["work"] == work
    assert abs(rl["peak"] - 152 * 64 * 2070e6 / 1e12) < 1e-9
    assert abs(rl["frac"] - work / 0.2629 / (152 * 64 * 2070e6)) < 1e-12
