"""Bit-exact parity with the oracle at every workload's stated size.

Each workload is built on the GPU through the C ABI at its full size, in
the launch configuration the benchmark uses (default options), and compared
word for word with the oracle run on the host: every bitmap word, zero
count, rank directory record and select sample; for the 4-ary tree every
per-digit-value directory record and digit sample; for the Huffman-shaped
tree the code lengths, codes, level lengths and level offsets too.  All
arithmetic is integer, so the tolerance is 0.

* 2^20 uint8 symbols, sigma 256, uniform: the balanced tree (and the
  matrix), plus 10^5 mixed access / rank / select queries (1% invalid)
  against the oracle's answers by definition (Section 2).
* 2^30 uint16 Zipf(1.1) symbols over 2^16: the wavelet matrix (Section
  4.3; 16 levels, 2^34 bitmap bits, 2^18 tiles per pass).
* 2^32 uint8 DNA-like symbols, sigma 5: the balanced binary tree (Section
  2; level positions past 2^32) and the 4-ary tree (Section 4.3 multiary;
  2^33 digit bits per level).
* 2^28 uint32 Zipf(1.0) symbols over 2^20: the Huffman-shaped tree
  (Section 4.3, arbitrary shapes) and the balanced tree of the same input.
* The batched workload (4096 sequences of log-uniform lengths, 2^31
  symbols in all) in one batched build: 300 sequences compared in full,
  the longest and the shortest among them.

The oracle runs at about 0.13 G symbol-levels/s on one core, so its builds
start in host threads (ctypes releases the GIL) before the GPU builds, and
the per-level directory and sample scans run in parallel.  Peak host memory
is about 120 GB (the oracle widens symbols to uint32 and keeps two copies)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (check_binary_dirs, check_binary_dirs_parallel, check_digit_dirs_parallel,
                      first_diff, from_dev_u64, oracle_pool, oracle_queries, queries_on, to_dev)

pytestmark = pytest.mark.gpu

SEED = synth.SEED_BASE


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


class Work:
    """Host inputs (pinned) of the large workloads and the oracle's builds of
    them, started in the pool as soon as each input exists."""

    def __init__(self):
        import torch
        pool = oracle_pool()
        # 2^30 uint16 Zipf(1.1) over 2^16 (the headline)
        n2 = 1 << 30
        self.pin2 = torch.empty(n2, dtype=torch.int16).pin_memory()
        synth.zipf(SEED + 2, n2, 1 << 16, 1.1, 2, addr=self.pin2.data_ptr())
        self.S2 = self.pin2.numpy().view(np.uint16)
        self.wm2 = pool.submit(oracle.wm_build, self.S2, 1 << 16)
        # 2^32 uint8 DNA-like text, sigma 5
        n3 = 1 << 32
        self.pin3 = torch.empty(n3, dtype=torch.uint8).pin_memory()
        synth.genome(SEED + 3, n3, addr=self.pin3.data_ptr())
        S3w = self.pin3.numpy().astype(np.uint32)   # one widened copy for both oracle builds
        self.wt3 = pool.submit(oracle.wt_build, S3w, 5)
        self.mwt3 = pool.submit(oracle.mwt_build, S3w, 5)
        del S3w
        # 2^28 uint32 Zipf(1.0) over 2^20
        n4 = 1 << 28
        self.pin4 = torch.empty(n4, dtype=torch.int32).pin_memory()
        synth.zipf(SEED + 4, n4, 1 << 20, 1.0, 4, addr=self.pin4.data_ptr())
        self.S4 = self.pin4.numpy().view(np.uint32)
        self.wt4 = pool.submit(oracle.wt_build, self.S4, 1 << 20)
        self.hf4 = pool.submit(self._huff_oracle, self.S4, 1 << 20)

    @staticmethod
    def _huff_oracle(S, sigma):
        hist = np.bincount(S, minlength=sigma).astype(np.uint64)
        ln, mx = oracle.huffman_lengths(hist, 32)
        code = oracle.canonical_codes(ln)
        bits, woff, nl = oracle.huff_wt_build(S, ln, code)
        return ln, mx, code, bits, woff, nl


@pytest.fixture(scope="module")
def work(wt):
    w = Work()
    yield w
    for f in (w.wm2, w.wt3, w.mwt3, w.wt4, w.hf4):
        f.cancel()


def _assert_words(got, exp, what):
    ok, msg = first_diff(got, exp)
    assert ok, f"{what}: {msg}"


def test_uniform_2e20_u8_sigma256_tree_and_1e5_queries(wt, work):
    n, sigma = 1 << 20, 256
    S = synth.uniform(SEED + 1, n, sigma, 1)
    d = to_dev(S)
    ob = oracle.wt_build(S, sigma)
    obm, ozm = oracle.wm_build(S, sigma)
    h = wt.wt_build(d, sigma)
    ex = h.export()
    _assert_words(ex.bits.reshape(ob.shape), ob, "balanced tree bitmaps")
    assert np.array_equal(ex.zeros, ozm)
    check_binary_dirs(ex, list(ob), [n] * ob.shape[0])
    q = 100000
    op, c, arg = synth.queries(SEED + 1, S, sigma, q)
    assert np.array_equal(queries_on(h, S, sigma, op, c, arg),
                          oracle_queries(S, sigma, op, c, arg))
    h.free()
    hm = wt.wm_build(d, sigma)
    exm = hm.export()
    _assert_words(exm.bits.reshape(obm.shape), obm, "wavelet matrix bitmaps")
    assert np.array_equal(exm.zeros, ozm)
    check_binary_dirs(exm, list(obm), [n] * obm.shape[0])
    assert np.array_equal(queries_on(hm, S, sigma, op, c, arg),
                          oracle_queries(S, sigma, op, c, arg))
    hm.free()


def _sampled_queries(h, S, rng, nsym=6, q=3000):
    """Access at random positions; rank and select for a few symbols, against
    positions found on the host."""
    import torch
    n = S.size
    i = rng.integers(0, n, q).astype(np.uint64)
    out = torch.empty(q, dtype=torch.int64, device="cuda")
    h.access(to_dev(i), out)
    assert np.array_equal(from_dev_u64(out), S[i.astype(np.int64)].astype(np.uint64))
    cs = np.unique(np.concatenate([S[rng.integers(0, n, nsym - 1)], [S[0]]]))
    for c in cs:
        pos = np.flatnonzero(S == c).astype(np.uint64)
        ii = rng.integers(0, n, q).astype(np.uint64)
        cc = np.full(q, c, np.uint32)
        h.rank(to_dev(cc), to_dev(ii), out)
        assert np.array_equal(from_dev_u64(out),
                              np.searchsorted(pos, ii, side="right").astype(np.uint64))
        kk = rng.integers(1, pos.size + 1, q).astype(np.uint64)
        h.select(to_dev(cc), to_dev(kk), out)
        assert np.array_equal(from_dev_u64(out), pos[(kk - 1).astype(np.int64)])


def test_headline_wm_2e30_u16_zipf_bit_exact(wt, work):
    n, sigma = 1 << 30, 1 << 16
    h = wt.wm_build(work.pin2.to("cuda"), sigma)
    ex = h.export()
    ob, oz = work.wm2.result()
    assert ex.levels == 16
    _assert_words(ex.bits.reshape(ob.shape), ob, "wavelet matrix bitmaps")
    assert np.array_equal(ex.zeros, oz)
    check_binary_dirs_parallel(ex, list(ob), [n] * 16)
    del ex, ob
    _sampled_queries(h, work.S2, np.random.default_rng(5))
    h.free()


def test_genome_2e32_u8_binary_and_4ary_bit_exact(wt, work):
    import torch
    n = 1 << 32
    d = work.pin3.to("cuda")
    h = wt.wt_build(d, 5)
    hm = wt.multiary_build(d, 5)
    del d
    torch.cuda.synchronize()
    ex = h.export()
    h.free()
    ob = work.wt3.result()
    assert ex.levels == 3 and ob.shape[0] == 3
    _assert_words(ex.bits.reshape(ob.shape), ob, "balanced tree bitmaps")
    check_binary_dirs_parallel(ex, list(ob), [n] * 3)
    del ex, ob
    exm = hm.export()
    hm.free()
    od = work.mwt3.result()
    assert exm.levels == 2 and od.shape[0] == 2
    _assert_words(exm.bits.reshape(od.shape), od, "4-ary digit levels")
    check_digit_dirs_parallel(exm, list(od), n)


def test_huffman_and_balanced_2e28_u32_sigma2e20_bit_exact(wt, work):
    n, sigma = 1 << 28, 1 << 20
    d = work.pin4.to("cuda")
    hh = wt.huff_wt_build(d, sigma)
    hb = wt.wt_build(d, sigma)
    exh = hh.export()
    hh.free()
    ln, mx, code, bits, woff, nl = work.hf4.result()
    assert np.array_equal(exh.code_len, ln) and np.array_equal(exh.code, code)
    assert exh.levels == mx and np.array_equal(exh.level_len, nl)
    assert np.array_equal(exh.level_off, woff)
    _assert_words(exh.bits, bits, "Huffman-shaped tree bitmaps")
    levels = [bits[int(woff[l]):int(woff[l + 1])] for l in range(mx)]
    check_binary_dirs_parallel(exh, levels, [int(x) for x in nl])
    del exh, bits, levels
    exb = hb.export()
    hb.free()
    ob = work.wt4.result()
    assert exb.levels == 20
    _assert_words(exb.bits.reshape(ob.shape), ob, "balanced tree bitmaps")
    check_binary_dirs_parallel(exb, list(ob), [n] * 20)


def _batch_seq_job(ex, S, sigma, i):
    ob, oz = oracle.wm_build(S, sigma)
    ok, msg = first_diff(ex.bits.reshape(ob.shape), ob)
    if not ok:
        return f"sequence {i} (n={S.size}, sigma={sigma}) bitmaps: {msg}"
    if not np.array_equal(ex.zeros, oz):
        return f"sequence {i} zero counts"
    try:
        check_binary_dirs(ex, list(ob), [S.size] * ob.shape[0])
    except AssertionError as e:
        return f"sequence {i}: {e}"
    return None


def test_batched_4096_sequences_bit_exact(wt, work):
    import torch
    m = 4096
    ln, sig, zf, sd, total = synth.batch_plan(SEED + 5, m, 10, 24, 1 << 31)
    assert total == int(ln.sum()) <= 1 << 31
    offs = np.zeros(m + 1, np.int64)
    for i in range(m):
        offs[i + 1] = offs[i] + (int(ln[i]) + 7) // 8 * 8
    pin = torch.empty(int(offs[-1]), dtype=torch.int16).pin_memory()
    base = pin.data_ptr()
    for i in range(m):
        n, s = int(ln[i]), int(sig[i])
        if zf[i]:
            synth.zipf(int(sd[i]), n, s, 1.1, 2, addr=base + 2 * int(offs[i]))
        else:
            synth.uniform(int(sd[i]), n, s, 2, addr=base + 2 * int(offs[i]))
    host = pin.numpy().view(np.uint16)
    d = pin.to("cuda")
    seqs = [d[int(offs[i]):int(offs[i]) + int(ln[i])] for i in range(m)]
    hs = wt.wm_batch_build(seqs, [int(x) for x in sig])
    rng = np.random.default_rng(6)
    check = sorted(set(rng.choice(m, 298, replace=False).tolist())
                   | {int(np.argmax(ln)), int(np.argmin(ln))})
    futs = []
    for i in check:
        S = host[int(offs[i]):int(offs[i]) + int(ln[i])]
        futs.append(oracle_pool().submit(_batch_seq_job, hs[i].export(), S, int(sig[i]), i))
    for h in hs:
        h.free()
    errs = [e for e in (f.result() for f in futs) if e]
    assert len(check) >= 300 and not errs, errs[:5]
