"""Multi-rank host logic on CPU: two gloo ranks (world size 2) shard the
batched workload and reduce timings, as the benchmark does under torchrun on
GPUs (one process per GPU, no data-path collective)."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1610_03524_gb300 import dist as wdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ln, _, _, _, _ = synth.batch_plan(synth.SEED_BASE + 5, 4096, 10, 24, 1 << 31)
        mine = wdist.shard(ln, world, rank)
        out = [None] * world
        dist.all_gather_object(out, mine)
        mx = wdist.max_over_ranks(10.0 + rank)
        sm = wdist.sum_over_ranks(float(sum(int(ln[i]) for i in mine)))
        q.put((rank, out, mx, sm))
    finally:
        dist.destroy_process_group()


def test_shard_and_reduce_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ln, _, _, _, total = synth.batch_plan(synth.SEED_BASE + 5, 4096, 10, 24, 1 << 31)
    for rank, shards, mx, sm in res:
        assert mx == 11.0
        assert sm == float(total)
        # both ranks see the same assignment; it covers every sequence once
        a, b = shards
        assert sorted(a + b) == list(range(4096)) and not set(a) & set(b)
        loads = [sum(int(ln[i]) for i in s) for s in shards]
        assert abs(loads[0] - loads[1]) <= int(max(ln))


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_partition_single_process(world):
    rng = np.random.default_rng(world)
    ln = rng.integers(1, 1000, size=257)
    parts = [wdist.shard(ln, world, r) for r in range(world)]
    allidx = sorted(i for p in parts for i in p)
    assert allidx == list(range(ln.size))
    loads = [int(ln[p].sum()) if p else 0 for p in parts]
    assert max(loads) - min(loads) <= int(ln.max())
    with pytest.raises(ValueError):
        wdist.shard(ln, world, world)
