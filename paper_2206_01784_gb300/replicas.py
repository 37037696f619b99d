"""Independent replicas across GPUs (one process per GPU).

A sort is one GPU's work; what spreads over several GPUs are independent
units (arrays of a workload, requests of a service, segments of a batch), so
multi-GPU here means sharding units across ranks with no collective on the
data path. torch.distributed is used only for host-side bookkeeping: the
barrier and max-over-ranks timing of the benchmark, and gathering per-rank
statistics.
"""
from __future__ import annotations

import heapq


def shard_round_robin(units: list, rank: int, world: int) -> list:
    """Units rank, rank + world, rank + 2*world, ..."""
    return list(units[rank::world])


def shard_balanced(sizes: list[int], world: int) -> list[list[int]]:
    """Greedy longest-first split of unit indices over ranks by size: each unit
    goes to the rank with the least work so far. Deterministic."""
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return [sorted(x) for x in out]


def _dist():
    import torch.distributed as dist

    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(x: float, device=None) -> float:
    import torch

    dist = _dist()
    if dist is None:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch

    dist = _dist()
    if dist is None:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_lists(values: list[float]) -> list[float]:
    """Concatenation of every rank's list (every rank receives it)."""
    dist = _dist()
    if dist is None:
        return list(values)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(values))
    return [v for part in out for v in part]
