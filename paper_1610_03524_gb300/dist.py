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


# ---------------------------------------------------------------------------
# Domain-decomposition merge across ranks (Section 4.2).  Rank k holds the
# structure of piece k of one sequence; the structure of the whole sequence is
# sharded by position: rank r owns positions [lo_r, lo_{r+1}) of every level,
# lo_r = floor(r n / R).  Every level of the whole lists its nodes in order
# and, inside a node, the pieces in order; so after one all-gather of the node
# sizes (R x (2^L - 1) counts) every rank computes the same plan, and rank k
# sends each of its (node, level) runs, cut at shard boundaries, to the owners.
# On one GPU the same plan runs as the wt_dd_merge kernels.
# ---------------------------------------------------------------------------
def dd_level_of(stride: int):
    """Level of each node column: level l holds columns 2^l - 1 .. 2^(l+1) - 2."""
    import numpy as np
    i = np.arange(stride, dtype=np.int64)
    return np.floor(np.log2(i + 1)).astype(np.int64)


def dd_plan(counts):
    """counts[k, 2^l - 1 + c]: size of node c of level l in piece k (nodes in
    the level's order: prefixes for a balanced tree, classes for a wavelet
    matrix).  Returns (src, dst): the start of each run in its piece's level
    and in the whole sequence's level."""
    import numpy as np
    counts = np.asarray(counts, dtype=np.int64)
    R, stride = counts.shape
    lev = dd_level_of(stride)
    first = (1 << lev) - 1            # first column of each column's level
    # inside a piece: exclusive prefix over the nodes of the level
    pre = np.cumsum(counts, axis=1) - counts
    src = pre - pre[:, first]
    # the whole: nodes in order, pieces in order inside a node
    tot = counts.sum(axis=0)
    gx = np.cumsum(tot) - tot
    g = gx - gx[first]
    dst = g[None, :] + (np.cumsum(counts, axis=0) - counts)
    return src, dst


def dd_shards(n: int, world: int):
    """Start of every rank's position range (world + 1 entries)."""
    return [r * n // world for r in range(world)] + [n]


def dd_messages(counts, src_rank: int, world: int):
    """Runs rank src_rank sends, per destination rank: arrays (level,
    source offset in its own level, destination offset in the receiver's
    shard, length), cut at the shard boundaries."""
    import numpy as np
    counts = np.asarray(counts, dtype=np.int64)
    src, dst = dd_plan(counts)
    n = int(counts[:, 0].sum())
    lo = np.asarray(dd_shards(n, world), dtype=np.int64)
    lev = dd_level_of(counts.shape[1])
    k = counts[src_rank]
    keep = k > 0
    L_, S_, D_, N_ = lev[keep], src[src_rank][keep], dst[src_rank][keep], k[keep]
    out = {r: ([], [], [], []) for r in range(world)}
    while L_.size:
        r = np.searchsorted(lo, D_, side="right") - 1     # owner of each run's first bit
        r = np.minimum(r, world - 1)
        take = np.minimum(N_, lo[r + 1] - D_)              # up to the owner's end
        for rr in np.unique(r):
            m = r == rr
            o = out[int(rr)]
            o[0].append(L_[m]); o[1].append(S_[m]); o[2].append(D_[m] - lo[rr]); o[3].append(take[m])
        rest = N_ > take                                   # the part past the boundary
        L_, S_, D_, N_ = L_[rest], S_[rest] + take[rest], D_[rest] + take[rest], N_[rest] - take[rest]
    res = {}
    for r, (a, b, c, d) in out.items():
        cat = (lambda x: np.concatenate(x) if x else np.zeros(0, np.int64))
        res[r] = (cat(a), cat(b), cat(c), cat(d))
    return res
