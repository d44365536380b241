"""Sharding of independent instances over ranks, run as two gloo ranks on CPU.

Every rank computes the same partition of the uneven batch, takes its share,
and the ranks check with collectives that each instance is owned by exactly
one rank, that the owned work adds up to the whole batch, and that the
greedy longest-first balance is within its 4/3 bound of the optimum.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1902_10078_gb300 import shard
from paper_1902_10078_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, count, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns, ls = W.batched_shapes(count)
        parts = shard.partition(ns, ls, world)
        mine = parts[rank]
        owned = torch.zeros(count, dtype=torch.int64)
        owned[mine] = 1
        dist.all_reduce(owned, op=dist.ReduceOp.SUM)
        work = torch.tensor([sum(shard.instance_cost(ns[i], ls[i]) for i in mine)], dtype=torch.float64)
        loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(loads, work)
        if rank == 0:
            out.put((owned.tolist(), [float(x) for x in loads]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_partition_two_gloo_ranks(world):
    count = 4096
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, count, q)) for r in range(world)]
    for p in procs:
        p.start()
    owned, loads = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert owned == [1] * count                      # every instance on exactly one rank
    ns, ls = W.batched_shapes(count)
    total = sum(shard.instance_cost(n, l) for n, l in zip(ns, ls))
    assert sum(loads) == pytest.approx(total, rel=0, abs=0.5)
    biggest = max(shard.instance_cost(n, l) for n, l in zip(ns, ls))
    assert max(loads) <= total / world + biggest     # LPT: within one instance of the mean


def test_partition_small_cases():
    assert shard.partition([5, 5, 5], [1, 1, 1], 1) == [[0, 1, 2]]
    parts = shard.partition([100, 1, 1, 1], [3, 3, 3, 3], 2)
    assert sorted(parts, key=len) == [[0], [1, 2, 3]]
    with pytest.raises(ValueError):
        shard.partition([1], [1], 0)
    # more ranks than instances: some ranks idle
    parts = shard.partition([3, 4], [1, 2], 4)
    assert sorted(sum(parts, [])) == [0, 1] and sum(1 for p in parts if not p) == 2
    assert sorted(shard.loads([3, 4], [1, 2], parts)) == [0, 0, 12, 36]


def _timing_rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 5.0 - rank, 2.5, 10.0 * rank]
        got = bench.max_over_ranks(mine, world, "cpu")
        out.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_bench_timings_take_the_slowest_rank():
    """bench.py reports, on every rank, the element-wise maximum of the ranks'
    timings (the job is as slow as its slowest rank)."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_timing_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert got[r] == [2.0, 5.0, 2.5, 10.0]
