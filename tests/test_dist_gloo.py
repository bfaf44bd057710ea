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


# ---------------------------------------------------------------------------
# domain-decomposition merge across ranks: the routing plan (dist.dd_*) with
# the pieces' level bits taken from the oracle and the bits moved by the
# test; each rank's assembled shard equals the same positions of the
# oracle's structure of the whole sequence
# ---------------------------------------------------------------------------
import oracle  # noqa: E402


def _rev(x, l):
    r = np.zeros_like(x)
    for i in range(l):
        r |= ((x >> i) & 1) << (l - 1 - i)
    return r


def _node_counts(P, L, wm):
    """Node sizes of every level of a piece, from its symbols."""
    out = []
    for l in range(L):
        t = (P.astype(np.int64) >> (L - l)) if l else np.zeros(P.size, np.int64)
        key = _rev(t, l) if wm else t
        out.append(np.bincount(key, minlength=1 << l)[: 1 << l])
    return np.concatenate(out).astype(np.int64)


def _level_bits(P, sigma, wm):
    L = oracle.levels(sigma)
    if P.size == 0:
        return [np.zeros(0, np.uint8) for _ in range(L)]
    ob = oracle.wm_build(P, sigma)[0] if wm else oracle.wt_build(P, sigma)
    return [np.unpackbits(ob[l].view(np.uint8), bitorder="little")[: P.size] for l in range(L)]


def _pieces(seed, n, sigma, world):
    S = synth.zipf(seed, n, sigma, 1.1, 2)
    rng = np.random.default_rng(seed)
    cut = [0, *sorted(rng.integers(0, n + 1, world - 1).tolist()), n]
    return S, [S[a:b] for a, b in zip(cut[:-1], cut[1:])]


def _assemble(msgs_to_me, bits_by_src, shard_len, L):
    out = [np.zeros(shard_len, np.uint8) for _ in range(L)]
    seen = [np.zeros(shard_len, np.int64) for _ in range(L)]
    for src, (lv, so, do, ln) in msgs_to_me.items():
        for l, a, b, m in zip(lv, so, do, ln):
            out[l][b:b + m] = bits_by_src[src][l][a:a + m]
            seen[l][b:b + m] += 1
    return out, seen


def _check_rank(S, sigma, wm, world, rank, msgs_to_me, bits_by_src):
    n, L = S.size, oracle.levels(sigma)
    lo = wdist.dd_shards(n, world)
    out, seen = _assemble(msgs_to_me, bits_by_src, lo[rank + 1] - lo[rank], L)
    full = _level_bits(S, sigma, wm)
    for l in range(L):
        assert np.all(seen[l] == 1), "runs tile the shard exactly once"
        assert np.array_equal(out[l], full[l][lo[rank]:lo[rank + 1]]), l


def _dd_rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for sigma, wm in ((4096, True), (300, False)):
            S, pieces = _pieces(71 + sigma, 60001, sigma, world)
            L = oracle.levels(sigma)
            mine = pieces[rank]
            counts = [None] * world
            dist.all_gather_object(counts, _node_counts(mine, L, wm))   # the one exchange of sizes
            counts = np.stack(counts)
            msgs = wdist.dd_messages(counts, rank, world)
            bits = _level_bits(mine, sigma, wm)
            payload = {r: [(int(l), bits[l][a:a + m].copy(), int(b))
                           for l, a, b, m in zip(*msgs[r])] for r in range(world)}
            got = [None] * world
            dist.all_gather_object(got, payload)                       # stands in for all-to-all
            to_me = {}
            bits_by_src = {}
            for src in range(world):
                segs = got[src][rank]
                lv = np.array([s[0] for s in segs], np.int64)
                do = np.array([s[2] for s in segs], np.int64)
                ln = np.array([s[1].size for s in segs], np.int64)
                # each received run is its own source array here
                bits_by_src[src] = {}
                so = np.zeros(len(segs), np.int64)
                for t, s in enumerate(segs):
                    bits_by_src[src].setdefault(s[0], [])
                    so[t] = sum(x.size for x in bits_by_src[src][s[0]])
                    bits_by_src[src][s[0]].append(s[1])
                bits_by_src[src] = {l: np.concatenate(v) for l, v in bits_by_src[src].items()}
                to_me[src] = (lv, so, do, ln)
            _check_rank(S, sigma, wm, world, rank, to_me, bits_by_src)
        q.put((rank, "ok"))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def test_dd_merge_routing_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dd_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res) == [(0, "ok"), (1, "ok")]


@pytest.mark.parametrize("world,sigma,wm", [(1, 256, True), (3, 77, True), (4, 1000, False),
                                            (5, 5, True)])
def test_dd_merge_routing_single_process(world, sigma, wm):
    S, pieces = _pieces(80 + world, 40003, sigma, world)
    L = oracle.levels(sigma)
    counts = np.stack([_node_counts(P, L, wm) for P in pieces])
    # the plan's run starts agree with each piece's own layout
    src, dst = wdist.dd_plan(counts)
    assert int(dst[-1, 0] + counts[-1, 0]) == S.size
    bits = [_level_bits(P, sigma, wm) for P in pieces]
    msgs = [wdist.dd_messages(counts, k, world) for k in range(world)]
    for r in range(world):
        _check_rank(S, sigma, wm, world, r, {k: msgs[k][r] for k in range(world)},
                    {k: bits[k] for k in range(world)})
