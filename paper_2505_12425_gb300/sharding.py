"""Multi-GPU host logic: the resampling path has no exchange step (images and tiles are
independent), so N GPUs run N replicas. A ragged batch or a request stream is split across
ranks by output pixels with a greedy longest-processing-time bin packing, and timings are
combined by taking the slowest rank. Only host-side bookkeeping lives here; every rank
launches its own share through the C ABI on its own GPU.
"""
from __future__ import annotations

import heapq


def shard_by_pixels(costs, world: int) -> list:
    """Assign item i (cost costs[i], e.g. output pixels) to one of `world` ranks.

    Largest items first, each to the currently least-loaded rank (ties: lower rank).
    Returns per-rank lists of item indices, each in increasing index order. Deterministic,
    so every rank computes the same plan without communicating.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(v) for v in out]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks of the default process group (the step time of
    the slowest rank); `value` itself when there is no process group."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
