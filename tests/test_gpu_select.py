"""GPU parity of the constant-time select directory (after Clark, Section 5.1
select; built with FLAG_SELECT_O1): every array equal to the oracle's
definition, and select answers equal to the oracle's select (bit-exact).

Inputs: the library's structures on cfg-like sequences, a bitvector with
long sparse stretches (sub-ranges of at least 2^16 bits keep all offsets),
and a bitvector of more than 2^32 bits whose first range spans more than
2^32 bits (the range keeps all positions)."""
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
    for l in range(ex.levels):
        nb = int(ex.level_len[l])
        lv = ex.level(l)
        for b in (0, 1):
            got = h.export_select(l, b)
            exp = oracle.clark(lv, nb, b)
            for g, e, name in zip(got, exp, ("desc", "sub", "sparse", "huge")):
                assert np.array_equal(g, e), f"level {l} bit {b} {name}"


CASES = [
    ("wm", "zipf", 1, 200000, 4096),
    ("wm", "uniform", 2, 70001, 5),
    ("wt", "zipf", 3, 150000, 1000),
    ("huff", "zipf", 4, 120000, 3000),
    ("wm", "uniform", 5, 1 << 20, 1 << 16),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-n{c[3]}-s{c[4]}")
def test_select_o1_structures(wt, case):
    kind, dist, seed, n, sigma = case
    S = synth.zipf(seed, n, sigma, 1.1, 2) if dist == "zipf" else synth.uniform(seed, n, sigma, 2)
    d = to_dev(S)
    fl = wt.FLAG_SELECT_O1
    h = {"wm": wt.wm_build, "wt": wt.wt_build}.get(kind, wt.huff_wt_build)(d, sigma, flags=fl)
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
