"""Multi-rank host logic of bench.py on CPU with the gloo backend (world
size 2): the timed region is the slowest rank's, and independent units are
dealt out without overlap.  One GPU per rank runs the same code with NCCL."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    got = bench.max_over_ranks(ms, dist)
    units = list(bench.shard(64, rank, world))
    out.put((rank, got, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert sorted(res[0][2] + res[1][2]) == list(range(64))
    assert not set(res[0][2]) & set(res[1][2])


def _deal_worker(rank, world, port, out):
    """Each rank deals the batched workload's 64 problems itself, as bench.py's
    batched run does; the ranks' shares must agree and cover every problem once."""
    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_2103_01691_b300 import inputs

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dims = inputs.batched_dims(64, seed=3)
    costs = [8.0 * float(np.prod(d)) * float(np.sum(d)) for d in dims]
    mine = bench.deal_by_cost(costs, world)[rank]
    load = sum(costs[i] for i in mine)
    out.put((rank, mine, load, max(costs), sum(costs)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_batched_dealing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_deal_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res[0][1] + res[1][1]) == list(range(64))
    assert not set(res[0][1]) & set(res[1][1])
    total, biggest = res[0][4], res[0][3]
    # greedy largest-first: no rank carries more than its share plus one problem
    assert max(r[2] for r in res) <= total / 2 + biggest


def test_deal_by_cost_balances():
    sys.path.insert(0, ROOT)
    import bench

    costs = [5.0, 9.0, 1.0, 7.0, 3.0, 3.0, 8.0]
    for world in (1, 2, 3, 7, 9):
        parts = bench.deal_by_cost(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)


def test_shard_covers_uneven_counts():
    sys.path.insert(0, ROOT)
    import bench

    for count in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            seen = [u for r in range(world) for u in bench.shard(count, r, world)]
            assert seen == list(range(count))
