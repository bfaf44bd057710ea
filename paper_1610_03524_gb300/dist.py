"""Multi-rank host logic: one process per GPU, launched by torchrun.

The wavelet-tree workloads shard as independent problems.  Each rank builds
its own sequences, and no collective touches the data path.  The only
collectives are the timing reduction (max over ranks) and the barriers
around the timed region.
"""
from __future__ import annotations

import heapq


def shard(lengths, world_size: int, rank: int) -> list[int]:
    """Indices of the sequences rank `rank` builds, out of sequences of the
    given lengths, for world_size ranks.

    Longest-first greedy assignment. Sequences are taken by decreasing length
    (ties by index), and each goes to the rank with the fewest symbols so far
    (ties to the lowest rank).  Every rank computes the same assignment
    without communication; the result is sorted.
    """
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    order = sorted(range(len(lengths)), key=lambda i: (-int(lengths[i]), i))
    heap = [(0, r) for r in range(world_size)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + int(lengths[i]), r))
    return sorted(mine)


def max_over_ranks(x: float) -> float:
    """The maximum of x over all ranks, or x itself outside a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    """The sum of x over all ranks, or x itself outside a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
