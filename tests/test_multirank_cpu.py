"""The multi-GPU host logic on CPU with two gloo ranks: every rank computes the same
pixel-balanced shard plan without communicating, the shards cover every item exactly
once, and the step time reported is the slowest rank's."""
from __future__ import annotations

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2505_12425_gb300 import inputs
from paper_2505_12425_gb300.sharding import max_over_ranks, shard_by_pixels


def test_shard_plan_is_a_balanced_partition():
    items = inputs.ragged_batch(1003, 256)
    costs = [it.h * it.w for it in items]
    for world in (1, 2, 3, 8):
        plan = shard_by_pixels(costs, world)
        flat = sorted(i for rank in plan for i in rank)
        assert flat == list(range(len(items)))
        loads = [sum(costs[i] for i in rank) for rank in plan]
        # greedy LPT: no rank exceeds the mean by more than the largest single item
        assert max(loads) - sum(loads) / world <= max(costs)
    with pytest.raises(ValueError):
        shard_by_pixels(costs, 0)


def test_max_over_ranks_without_a_group_is_identity():
    assert max_over_ranks(3.5) == 3.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = inputs.ragged_batch(1003, 64)
        costs = [it.h * it.w for it in items]
        plan = shard_by_pixels(costs, world)
        mine = plan[rank]
        # the "step time" of a rank: its share of the pixels
        t = max_over_ranks(float(sum(costs[i] for i in mine)), dist)
        got = [None] * world
        dist.all_gather_object(got, mine)
        q.put((rank, mine, got, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_plan_and_max():
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
    res.sort()
    items = inputs.ragged_batch(1003, 64)
    costs = [it.h * it.w for it in items]
    expect = shard_by_pixels(costs, world)
    for rank, mine, got, t in res:
        assert mine == expect[rank]
        assert got == expect                          # every rank holds the same plan
        assert t == max(sum(costs[i] for i in r) for r in expect)
    assert sorted(i for r in expect for i in r) == list(range(64))
