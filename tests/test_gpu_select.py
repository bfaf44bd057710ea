"""GPU parity of the constant-time select directory (after Clark, Section 5.1
select; per digit value on 4-ary digit levels, Section 5.2 generalized
select; built with FLAG_SELECT_O1): every array equal to the oracle's
definition, and select answers equal to the oracle's select (bit-exact).

Inputs: the library's structures on cfg-like sequences, a bitvector and a
4-ary tree with long sparse stretches (sub-ranges of at least 2^16 positions
keep all offsets), and a bitvector and a 4-ary tree of more than 2^32
positions whose first range spans more than 2^32 (the range keeps all
positions)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import UMAX, from_dev_u64, oracle_queries, queries_on, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03524_gb300 as m
    m.load_library()
    return m


def check_arrays(h, ex):
    dig = ex.bits_per_elem == 2
    for l in range(ex.levels):
        nb = int(ex.level_len[l])
        lv = ex.level(l)
        for b in range(4 if dig else 2):
            got = h.export_select(l, b)
            exp = oracle.clark_digits(lv, nb, b) if dig else oracle.clark(lv, nb, b)
            for g, e, name in zip(got, exp, ("desc", "sub", "sparse", "huge")):
                assert np.array_equal(g, e), f"level {l} value {b} {name}"


CASES = [
    ("wm", "zipf", 1, 200000, 4096),
    ("wm", "uniform", 2, 70001, 5),
    ("wt", "zipf", 3, 150000, 1000),
    ("huff", "zipf", 4, 120000, 3000),
    ("wm", "uniform", 5, 1 << 20, 1 << 16),
    ("multi", "zipf", 6, 150000, 1000),
    ("multi", "uniform", 7, 1 << 20, 4),
    ("multi", "zipf", 8, 200001, 77),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-n{c[3]}-s{c[4]}")
def test_select_o1_structures(wt, case):
    kind, dist, seed, n, sigma = case
    S = synth.zipf(seed, n, sigma, 1.1, 2) if dist == "zipf" else synth.uniform(seed, n, sigma, 2)
    d = to_dev(S)
    fl = wt.FLAG_SELECT_O1
    h = {"wm": wt.wm_build, "wt": wt.wt_build, "multi": wt.multiary_build}.get(
        kind, wt.huff_wt_build)(d, sigma, flags=fl)
    ex = h.export()
    check_arrays(h, ex)
    op, c, x = synth.queries(40 + seed, S, sigma, 20000)
    sel = op == 2
    got = queries_on(h, S, sigma, op[sel], c[sel], x[sel])
    assert np.array_equal(got, oracle_queries(S, sigma, op[sel], c[sel], x[sel]))
    h.free()


def _bitvector(nbits, ones):
    words = np.zeros(oracle.level_words(nbits), dtype=np.uint64)
    ones = np.asarray(ones, dtype=np.uint64)
    np.bitwise_or.at(words, (ones >> np.uint64(6)).astype(np.int64),
                     np.left_shift(np.uint64(1), ones & np.uint64(63)))
    return words


def _rs_select(wt, h, bit, ks):
    import torch
    c = to_dev(np.full(ks.size, bit, np.uint32))
    k = to_dev(ks.astype(np.uint64))
    o = torch.empty(ks.size, dtype=torch.int64, device="cuda")
    h.select(c, k, o)
    return from_dev_u64(o)


def test_select_o1_sparse_stretches(wt):
    # dense stretches, and stretches with one 1 every 300 bits (256 ones span
    # 76800 bits >= 2^16)
    rng = np.random.default_rng(11)
    nbits = 1 << 24
    parts = []
    p = 0
    while p < nbits:
        if (p // (1 << 20)) % 2 == 0:
            seg = np.arange(p, min(p + (1 << 20), nbits), 300)
        else:
            m = min(1 << 20, nbits - p)
            seg = p + np.nonzero(rng.random(m) < 0.5)[0]
        parts.append(seg)
        p += 1 << 20
    ones = np.concatenate(parts).astype(np.uint64)
    words = _bitvector(nbits, ones)
    d = to_dev(words)
    h = wt.rs_build(d, nbits, flags=wt.FLAG_SELECT_O1)
    ex = h.export()
    check_arrays(h, ex)
    desc, _, sparse, _ = h.export_select(0, 1)
    assert sparse.size > 0 and any((int(v) >> 40) & 0xFFFF for v in desc)
    for bit in (0, 1):
        pos = ones if bit else np.setdiff1d(np.arange(nbits, dtype=np.uint64), ones)
        ks = np.unique(np.concatenate([np.arange(1, pos.size + 1, 97), [pos.size]])).astype(np.uint64)
        assert np.array_equal(_rs_select(wt, h, bit, ks), pos[(ks - 1).astype(np.int64)])
    h.free()


def test_select_o1_huge_range(wt):
    """A bitvector of 2^32 + 2^20 bits: its first 4096 ones are at the start,
    the next ones only past 2^32, so range 0 of the ones spans more than 2^32
    bits and keeps all 4096 positions."""
    nbits = (1 << 32) + (1 << 20)
    first = np.arange(0, 3 * 4096, 3, dtype=np.uint64)
    tail = (1 << 32) + np.arange(0, 1 << 19, 7, dtype=np.uint64)
    ones = np.concatenate([first, tail])
    words = _bitvector(nbits, ones)
    d = to_dev(words)
    del words
    h = wt.rs_build(d, nbits, flags=wt.FLAG_SELECT_O1)
    desc, sub, sparse, huge = h.export_select(0, 1)
    assert int(desc[0]) >> 63 == 1 and int(desc[0]) & ((1 << 63) - 1) == 0
    assert np.array_equal(huge[:4096], first)
    assert desc.size == (ones.size + 4095) // 4096
    ks = np.concatenate([np.arange(1, ones.size + 1, 5), [ones.size]]).astype(np.uint64)
    assert np.array_equal(_rs_select(wt, h, 1, ks), ones[(ks - 1).astype(np.int64)])
    # zeros: the k-th zero by counting the ones before it
    nz = nbits - ones.size
    kz = np.unique(np.concatenate([np.linspace(1, nz, 5000).astype(np.uint64), [1, nz]]))
    # position p of the k-th zero: smallest p with p + 1 - (ones <= p) = k
    lo = kz - np.uint64(1)
    for _ in range(200):  # fixed point from below: p = k - 1 + #(ones <= p)
        nxt = kz - np.uint64(1) + np.searchsorted(ones, lo, side="right").astype(np.uint64)
        if np.array_equal(nxt, lo):
            break
        lo = nxt
    assert np.array_equal(_rs_select(wt, h, 0, kz), lo)
    h.free()


def test_select_o1_multiary_sparse_stretches(wt):
    """A 4-ary tree over sigma = 4 (one digit level = the symbols): stretches
    where value 3 occurs once every 300 positions give it long sub-ranges."""
    rng = np.random.default_rng(12)
    n = 1 << 22
    x = rng.integers(0, 3, n).astype(np.uint8)
    sparse = (np.arange(n) // (1 << 19)) % 2 == 0
    x[sparse & (np.arange(n) % 300 == 7)] = 3
    x[~sparse & (rng.random(n) < 0.3)] = 3
    h = wt.multiary_build(to_dev(x), 4, flags=wt.FLAG_SELECT_O1)
    ex = h.export()
    check_arrays(h, ex)
    desc, _, sp, _ = h.export_select(0, 3)
    assert sp.size > 0 and any((int(v) >> 40) & 0xFFFF for v in desc)
    for d in range(4):
        pos = np.flatnonzero(x == d).astype(np.uint64)
        ks = np.unique(np.concatenate([np.arange(1, pos.size + 1, 97), [pos.size]])).astype(np.uint64)
        assert np.array_equal(_sel(wt, h, d, ks), pos[(ks - 1).astype(np.int64)])
    h.free()


def _sel(wt, h, c, ks):
    import torch
    o = torch.empty(ks.size, dtype=torch.int64, device="cuda")
    h.select(to_dev(np.full(ks.size, c, np.uint32)), to_dev(ks.astype(np.uint64)), o)
    return from_dev_u64(o)


def test_select_o1_multiary_huge_range(wt):
    """4-ary tree of 2^32 + 2^20 symbols over sigma = 4: value 3 occurs 4096
    times at the start and again only past 2^32, so its first range spans
    more than 2^32 digits and keeps all 4096 positions."""
    import torch
    n = (1 << 32) + (1 << 20)
    first = np.arange(0, 3 * 4096, 3, dtype=np.int64)
    tail = (1 << 32) + np.arange(0, 1 << 19, 7, dtype=np.int64)
    pin = torch.zeros(n, dtype=torch.uint8).pin_memory()
    host = pin.numpy()
    host[first] = 3
    host[tail] = 3
    host[(1 << 31):(1 << 31) + (1 << 20):5] = 1  # a few ones in the gap
    d = pin.to("cuda")
    h = wt.multiary_build(d, 4, flags=wt.FLAG_SELECT_O1)
    desc, sub, sp, huge = h.export_select(0, 3)
    assert int(desc[0]) >> 63 == 1 and int(desc[0]) & ((1 << 63) - 1) == 0
    pos3 = np.concatenate([first, tail]).astype(np.uint64)
    assert np.array_equal(huge[:4096], pos3[:4096])
    assert desc.size == (pos3.size + 4095) // 4096
    ks = np.concatenate([np.arange(1, pos3.size + 1, 5), [pos3.size]]).astype(np.uint64)
    assert np.array_equal(_sel(wt, h, 3, ks), pos3[(ks - 1).astype(np.int64)])
    pos1 = np.arange(1 << 31, (1 << 31) + (1 << 20), 5, dtype=np.uint64)
    k1 = np.arange(1, pos1.size + 1, 3, dtype=np.uint64)
    assert np.array_equal(_sel(wt, h, 1, k1), pos1[(k1 - 1).astype(np.int64)])
    # zeros: the k-th zero by counting the non-zeros before it
    nz_pos = np.sort(np.concatenate([pos3, pos1]))
    nz = n - nz_pos.size
    kz = np.unique(np.concatenate([np.linspace(1, nz, 3000).astype(np.uint64), [1, nz]]))
    lo = kz - np.uint64(1)
    for _ in range(200):  # fixed point from below: p = k - 1 + #(non-zeros <= p)
        nxt = kz - np.uint64(1) + np.searchsorted(nz_pos, lo, side="right").astype(np.uint64)
        if np.array_equal(nxt, lo):
            break
        lo = nxt
    assert np.array_equal(_sel(wt, h, 0, kz), lo)
    h.free()
