"""GPU parity: every output of the CUDA path, through the C ABI, against the
CPU oracle on the same seeded inputs.  All arithmetic is integer, so every
bitmap word, directory record, select sample, zero count and query answer
must be bit-exact (tolerance 0).

Sizes span several 4096-symbol tiles with ragged tails; edge cases cover
empty, single-symbol, sigma in {1, 2, 3, 5, 2^k, 2^k+1}, constant and sorted
inputs, every tau, and a symbol >= sigma."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import (check_binary_dirs, from_dev_u64, oracle_queries, queries_on, to_dev)

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


def gen(kind, seed, n, sigma, width):
    if kind == "uniform":
        return synth.uniform(seed, n, sigma, width)
    if kind == "zipf":
        return synth.zipf(seed, n, sigma, 1.1, width)
    if kind == "const":
        return np.full(n, sigma - 1, dtype={1: np.uint8, 2: np.uint16, 4: np.uint32}[width])
    if kind == "sorted":
        return (np.arange(n, dtype=np.uint64) * sigma // max(n, 1)).astype(
            {1: np.uint8, 2: np.uint16, 4: np.uint32}[width])
    raise ValueError(kind)


CASES = [
    # kind, seed, n, sigma, width
    ("uniform", 1, 1, 2, 1),
    ("uniform", 2, 63, 5, 1),
    ("uniform", 3, 64, 3, 1),
    ("uniform", 4, 65, 8, 1),
    ("uniform", 5, 2047, 256, 1),
    ("uniform", 6, 2049, 257, 2),
    ("zipf", 7, 8191, 1000, 2),
    ("zipf", 8, 8192, 4096, 2),
    ("zipf", 9, 8193, 65536, 2),
    ("uniform", 10, 50000, 1, 1),
    ("const", 11, 30000, 77, 1),
    ("sorted", 12, 40000, 300, 2),
    ("zipf", 13, 100003, 65536, 2),
    ("uniform", 14, 70001, 1 << 20, 4),
    ("zipf", 15, 123457, 5, 1),
    ("uniform", 16, 1 << 18, 256, 1),
]


def build_case(wt, case, fn, **kw):
    kind, seed, n, sigma, width = case
    S = gen(kind, seed, n, sigma, width)
    h = fn(to_dev(S), sigma, **kw)
    return S, sigma, h


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-n{c[2]}-s{c[3]}-w{c[4]}")
def test_wm_parity(wt, case):
    S, sigma, h = build_case(wt, case, wt.wm_build)
    ex = h.export()
    ob, oz = oracle.wm_build(S, sigma)
    assert ex.levels == ob.shape[0]
    assert np.array_equal(ex.bits.reshape(ob.shape), ob)
    assert np.array_equal(ex.zeros, oz)
    check_binary_dirs(ex, list(ob), [S.size] * ob.shape[0])
    h.free()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-n{c[2]}-s{c[3]}-w{c[4]}")
def test_wt_parity(wt, case):
    S, sigma, h = build_case(wt, case, wt.wt_build)
    ex = h.export()
    ob = oracle.wt_build(S, sigma)
    assert np.array_equal(ex.bits.reshape(ob.shape), ob)
    ones = ob.copy()
    check_binary_dirs(ex, list(ob), [S.size] * ob.shape[0])
    # zero counts of the balanced tree equal those of the matrix (same bits per level)
    _, oz = oracle.wm_build(S, sigma)
    assert np.array_equal(ex.zeros, oz)
    del ones
    h.free()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-n{c[2]}-s{c[3]}-w{c[4]}")
def test_multiary_parity(wt, case):
    S, sigma, h = build_case(wt, case, wt.multiary_build)
    ex = h.export()
    od = oracle.mwt_build(S, sigma)
    assert ex.levels == od.shape[0]
    assert np.array_equal(ex.bits.reshape(od.shape), od)
    for b in range(od.shape[0]):
        assert np.array_equal(ex.level_dir(b), oracle.mwt_dir(od[b], S.size))
        # select samples of every digit value (Section 5.2 generalized select)
        for d in range(4):
            assert np.array_equal(ex.samples(b, d), oracle.digit_samples(od[b], S.size, d)), (b, d)
    h.free()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-n{c[2]}-s{c[3]}-w{c[4]}")
def test_huffman_parity(wt, case):
    S, sigma, h = build_case(wt, case, wt.huff_wt_build)
    ex = h.export()
    hist = np.bincount(S.astype(np.int64), minlength=sigma).astype(np.uint64)
    ln, mx = oracle.huffman_lengths(hist, 32)
    code = oracle.canonical_codes(ln)
    assert np.array_equal(ex.code_len, ln) and np.array_equal(ex.code, code)
    bits, woff, nl = oracle.huff_wt_build(S, ln, code)
    assert ex.levels == mx and np.array_equal(ex.level_len, nl)
    assert np.array_equal(ex.level_off, woff)
    assert np.array_equal(ex.bits, bits)
    levels = [bits[int(woff[l]):int(woff[l + 1])] for l in range(mx)]
    check_binary_dirs(ex, levels, [int(x) for x in nl])
    h.free()


@pytest.mark.parametrize("kind", ["flat", "mixed", "deep"])
def test_huffman_caller_lengths(wt, kind):
    """Caller-given code lengths, incomplete codes included (Kraft sum < 1):
    the tree follows the canonical codes of those lengths (Section 4.3 takes
    the shape as codewords)."""
    rng = np.random.default_rng({"flat": 1, "mixed": 2, "deep": 3}[kind])
    sigma = 700
    S = synth.zipf(50 + len(kind), 90001, sigma, 1.1, 2)
    present = np.bincount(S.astype(np.int64), minlength=sigma) > 0
    if kind == "flat":
        ln = np.full(sigma, 11, np.uint8)            # Kraft 700/2048
    elif kind == "mixed":
        ln = rng.integers(10, 15, sigma).astype(np.uint8)
    else:
        ln = np.full(sigma, 14, np.uint8)            # 31/32 + 400/2^14 + 295/2^30 < 1
        ln[:5] = [1, 2, 3, 4, 5]
        ln[5:300] = 30                               # long codes: 30 levels
    ln[~present & (rng.random(sigma) < 0.5)] = 0     # some absent symbols get no code
    assert float(np.sum(np.ldexp(1.0, -ln[ln > 0].astype(int)))) <= 1.0
    h = wt.huff_wt_build(to_dev(S), sigma, code_len=ln)
    ex = h.export()
    code = oracle.canonical_codes(ln)
    assert np.array_equal(ex.code_len, ln) and np.array_equal(ex.code, code)
    bits, woff, nl = oracle.huff_wt_build(S, ln, code)
    assert ex.levels == int(ln.max()) and np.array_equal(ex.level_len, nl)
    assert np.array_equal(ex.level_off, woff)
    assert np.array_equal(ex.bits, bits)
    levels = [bits[int(woff[l]):int(woff[l + 1])] for l in range(int(ln.max()))]
    check_binary_dirs(ex, levels, [int(x) for x in nl])
    h.free()


@pytest.mark.parametrize("tau", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tau_invariance(wt, tau):
    S = synth.zipf(21, 30011, 3000, 1.1, 2)
    ob, oz = oracle.wm_build(S, 3000)
    tb = oracle.wt_build(S, 3000)
    h = wt.wm_build(to_dev(S), 3000, tau=tau)
    assert np.array_equal(h.export().bits.reshape(ob.shape), ob)
    h.free()
    h = wt.wt_build(to_dev(S), 3000, tau=tau)
    assert np.array_equal(h.export().bits.reshape(tb.shape), tb)
    h.free()
    if tau % 2 == 0:
        h = wt.multiary_build(to_dev(S), 3000, tau=tau)
        assert np.array_equal(h.export().bits.reshape(-1), oracle.mwt_build(S, 3000).reshape(-1))
        h.free()
    h = wt.huff_wt_build(to_dev(S), 3000, tau=tau)
    hist = np.bincount(S.astype(np.int64), minlength=3000).astype(np.uint64)
    ln, _ = oracle.huffman_lengths(hist, 32)
    bits, _, _ = oracle.huff_wt_build(S, ln, oracle.canonical_codes(ln))
    assert np.array_equal(h.export().bits, bits)
    h.free()


@pytest.mark.parametrize("tile", [2048, 4096, 8192])
@pytest.mark.parametrize("ctas", [0, 1, 3])
def test_tile_sizes(wt, tile, ctas):
    """Wavelet matrices at every supported tile size (the paper's K = n / tile
    sub-problems, Section 4.2) and CTA count: bits, zero counts, directories
    and samples equal the oracle's; sizes span several tiles with a ragged
    tail, one pass and two passes."""
    for (seed, n, sigma, tau) in [(61, 100003, 65536, 8), (62, 3 * 8192 + 5, 300, 0),
                                  (63, (1 << 20) + 17, 256, 3), (64, 1000, 1 << 20, 5)]:
        S = synth.zipf(seed, n, sigma, 1.1, 2 if sigma <= 65536 else 4)
        ob, oz = oracle.wm_build(S, sigma)
        h = wt.wm_build(to_dev(S), sigma, tau=tau, ctas_per_sm=ctas, tile_symbols=tile)
        ex = h.export()
        assert np.array_equal(ex.bits.reshape(ob.shape), ob), (seed, tile, ctas)
        assert np.array_equal(ex.zeros, oz)
        check_binary_dirs(ex, list(ob), [n] * ob.shape[0])
        h.free()


@pytest.mark.parametrize("ctas", [1, 2])
def test_ctas_invariance(wt, ctas):
    S = synth.uniform(31, 200001, 65536, 2)
    ob, _ = oracle.wm_build(S, 65536)
    h = wt.wm_build(to_dev(S), 65536, ctas_per_sm=ctas)
    assert np.array_equal(h.export().bits.reshape(ob.shape), ob)
    h.free()


@pytest.mark.parametrize("kind", ["wm", "wt", "multi", "huff"])
@pytest.mark.parametrize("case", [("zipf", 41, 100000, 256, 1), ("uniform", 42, 5000, 1000, 2),
                                  ("zipf", 43, 77777, 65536, 2), ("uniform", 44, 3000, 5, 1),
                                  ("uniform", 45, 999, 1, 1)],
                         ids=lambda c: f"{c[0]}-n{c[2]}-s{c[3]}")
def test_queries(wt, kind, case):
    fn = {"wm": wt.wm_build, "wt": wt.wt_build, "multi": wt.multiary_build,
          "huff": wt.huff_wt_build}[kind]
    S, sigma, h = build_case(wt, case, fn)
    op, c, arg = synth.queries(7, S, sigma, 20000)
    got = queries_on(h, S, sigma, op, c, arg)
    exp = oracle_queries(S, sigma, op, c, arg)
    bad = np.nonzero(got != exp)[0]
    assert bad.size == 0, f"{bad.size} mismatches, first op={op[bad[0]]} c={c[bad[0]]} arg={arg[bad[0]]} got={got[bad[0]]} exp={exp[bad[0]]}"
    h.free()


@pytest.mark.parametrize("nbits,seed", [(1, 1), (64, 2), (2047, 3), (2048, 4), (100001, 5),
                                        (1 << 20, 6)])
def test_rs_parity(wt, nbits, seed):
    import torch
    W = (nbits + 63) // 64
    words = synth.words(seed, W)
    if seed % 2:
        words &= synth.words(seed + 9, W)  # sparser ones
    if nbits % 64:
        words[-1] &= np.uint64((1 << (nbits % 64)) - 1)
    d = to_dev(words)
    h = wt.rs_build(d, nbits)
    ex = h.export()
    full = np.zeros(oracle.level_words(nbits), dtype=np.uint64)
    full[:W] = words
    check_binary_dirs(ex, [full], [nbits])
    bits01 = np.array([(int(full[i >> 6]) >> (i & 63)) & 1 for i in range(nbits)], dtype=np.uint32)
    op, c, arg = synth.queries(8, bits01, 2, 4000)
    got = queries_on(h, bits01, 2, op, c, arg)
    exp = oracle_queries(bits01, 2, op, c, arg)
    assert np.array_equal(got, exp)
    h.free()
    del torch


def test_symbol_out_of_range(wt):
    S = synth.uniform(51, 10000, 100, 1)
    S[1234] = 200
    for fn in (wt.wm_build, wt.wt_build, wt.multiary_build, wt.huff_wt_build):
        h = fn(to_dev(S), 100)
        with pytest.raises(wt.WaveletError) as ei:
            h.sync()
        assert ei.value.status == 2
        h.free()


def test_huffman_build_is_asynchronous(wt):
    """huff_wt_build returns once the input's copy is enqueued: the caller may
    overwrite its input right after the stream passes the copy, several
    builds may be in flight, and each handle's first use waits for its build
    (queries on another stream are ordered after it)."""
    import torch
    seqs = [synth.zipf(60 + i, 200003 + 31 * i, 5000, 1.0, 4) for i in range(3)]
    d = torch.empty(max(S.size for S in seqs), dtype=torch.int32, device="cuda")
    hs = []
    for S in seqs:
        d[:S.size].copy_(torch.from_numpy(S.view(np.int32)).to("cuda"))
        hs.append(wt.huff_wt_build(d[:S.size], 5000))   # d is overwritten by the next copy
    other = torch.cuda.Stream()
    for S, h in zip(seqs, hs):
        hist = np.bincount(S.astype(np.int64), minlength=5000).astype(np.uint64)
        ln, _ = oracle.huffman_lengths(hist, 32)
        bits, woff, nl = oracle.huff_wt_build(S, ln, oracle.canonical_codes(ln))
        q = 2000
        op, c, arg = synth.queries(7, S, 5000, q)
        m = op == 1
        out = torch.empty(int(m.sum()), dtype=torch.int64, device="cuda")
        h.rank(to_dev(c[m]), to_dev(arg[m]), out, stream=other)
        other.synchronize()
        assert np.array_equal(from_dev_u64(out), oracle.rank(S, 5000, c[m], arg[m]))
        assert np.array_equal(h.export().bits, bits)
        h.free()


def test_huffman_invalid_caller_lengths_reported_on_use(wt):
    S = synth.uniform(52, 5000, 50, 1)
    ln = np.full(50, 6, np.uint8)
    ln[S[0]] = 0  # a present symbol without a code
    h = wt.huff_wt_build(to_dev(S), 50, code_len=ln)
    with pytest.raises(wt.WaveletError) as ei:
        h.sync()
    assert ei.value.status == 1
    h.free()
    ln = np.full(50, 2, np.uint8)  # Kraft sum 50/4 > 1
    h = wt.huff_wt_build(to_dev(S), 50, code_len=ln)
    with pytest.raises(wt.WaveletError) as ei:
        h.export()
    assert ei.value.status == 1
    h.free()


def test_empty_and_invalid(wt):
    import torch
    e = torch.empty(0, dtype=torch.uint8, device="cuda")
    for fn in (wt.wm_build, wt.wt_build, wt.multiary_build, wt.huff_wt_build):
        h = fn(e, 10)
        ex = h.export()
        assert ex.n == 0
        h.free()
    with pytest.raises(wt.WaveletError):
        wt.wm_build(e, 0)
    with pytest.raises(wt.WaveletError):
        wt.multiary_build(e, 10, degree=8)


def test_repeated_builds_identical(wt):
    S = synth.zipf(61, 300007, 65536, 1.1, 2)
    d = to_dev(S)
    first = None
    for _ in range(3):
        h = wt.wm_build(d, 65536)
        b = h.export().bits
        h.free()
        if first is None:
            first = b
        assert np.array_equal(b, first)


@pytest.mark.parametrize("tau", [3, 5, 6])
@pytest.mark.parametrize("seed,n,sigma", [(21, 30011, 3000), (22, 100000, 70000), (23, 20000, 40)])
def test_huffman_tau_levels(wt, tau, seed, n, sigma):
    S = synth.zipf(seed, n, sigma, 1.1, 2 if sigma <= 65536 else 4)
    hist = np.bincount(S.astype(np.int64), minlength=sigma).astype(np.uint64)
    ln, mx = oracle.huffman_lengths(hist, 32)
    bits, woff, nl = oracle.huff_wt_build(S, ln, oracle.canonical_codes(ln))
    h = wt.huff_wt_build(to_dev(S), sigma, tau=tau)
    ex = h.export()
    for l in range(mx):
        a, b = ex.level(l), bits[int(woff[l]):int(woff[l + 1])]
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, (f"level {l} of {mx}: {bad.size} words differ, first {bad[0]} "
                               f"of {a.size}, got {int(a[bad[0]]):016x} exp {int(b[bad[0]]):016x}")
    h.free()


@pytest.mark.parametrize("sigma,off", [(5, 3), (2, 0), (8, 7), (3, 1)])
def test_tiny_alphabet_histogram(wt, sigma, off):
    """Byte sequences over at most 8 values (counted four bytes to a word
    where the start is 16-byte aligned, one by one elsewhere): the balanced
    tree, which plans from the full histogram, equals the oracle's, aligned
    and not; a byte >= sigma in the tail is reported."""
    S = synth.uniform(310 + sigma, 70001 + off, sigma, 1)
    Sv = S[off:]
    h = wt.wt_build(to_dev(S)[off:], sigma)
    ob = oracle.wt_build(Sv, sigma)
    assert np.array_equal(h.export().bits.reshape(ob.shape), ob)
    h.free()
    bad = S.copy()
    bad[-2] = sigma
    h = wt.wt_build(to_dev(bad), sigma)
    with pytest.raises(wt.WaveletError) as ei:
        h.sync()
    assert ei.value.status == 2
    h.free()


@pytest.mark.parametrize("width,off", [(1, 5), (2, 3), (4, 1)])
def test_unaligned_input_pointer(wt, width, off):
    """A sequence that starts at an address not 16-byte aligned (a slice of a
    larger buffer) takes the scalar load paths and builds the same bits."""
    sigma = {1: 200, 2: 40000, 4: 70000}[width]
    S = synth.uniform(300 + width, 20000 + off, sigma, width)
    d = to_dev(S)[off:]
    Sv = S[off:]
    for fn in (wt.wm_build, wt.wt_build):
        h = fn(d, sigma)
        ex = h.export()
        ob = oracle.wm_build(Sv, sigma)[0] if fn is wt.wm_build else oracle.wt_build(Sv, sigma)
        assert np.array_equal(ex.bits.reshape(ob.shape), ob)
        h.free()
    hs = wt.wm_batch_build([d, to_dev(S)[1:]], [sigma, sigma])
    ob, _ = oracle.wm_build(Sv, sigma)
    assert np.array_equal(hs[0].export().bits.reshape(ob.shape), ob)
    ob, _ = oracle.wm_build(S[1:], sigma)
    assert np.array_equal(hs[1].export().bits.reshape(ob.shape), ob)


@pytest.mark.parametrize("case", [("zipf", 81, 12289, 65536, 2), ("uniform", 82, 4097, 200, 1),
                                  ("uniform", 83, 30001, 1 << 20, 4), ("zipf", 84, 1, 7, 2)],
                         ids=lambda c: f"{c[0]}-n{c[2]}-s{c[3]}-w{c[4]}")
@pytest.mark.parametrize("pinned", [True, False])
def test_wm_build_host_parity(wt, case, pinned):
    """The host-memory build (the library copies the sequence in on the
    stream) gives the oracle's wavelet matrix, from page-locked and from
    pageable memory."""
    import torch
    kind, seed, n, sigma, width = case
    S = gen(kind, seed, n, sigma, width)
    t = torch.from_numpy(S.view({1: np.uint8, 2: np.int16, 4: np.int32}[width]))
    if pinned:
        t = t.pin_memory()
    h = wt.wm_build_host(t, sigma)
    ex = h.export()
    ob, oz = oracle.wm_build(S, sigma)
    assert ex.levels == ob.shape[0]
    assert np.array_equal(ex.bits.reshape(ob.shape), ob)
    assert np.array_equal(ex.zeros, oz)
    check_binary_dirs(ex, list(ob), [S.size] * ob.shape[0])
    h.free()


def test_wm_build_host_errors(wt):
    import torch
    S = synth.uniform(85, 5000, 100, 2)
    # a symbol >= sigma: reported by the handle, as for wm_build
    h = wt.wm_build_host(S, 50)
    with pytest.raises(wt.WaveletError) as e:
        h.sync()
    assert e.value.status == 2
    h.free()
    with pytest.raises(wt.WaveletError):
        wt.wm_build_host(S, 0)
    with pytest.raises(ValueError):
        wt.wm_build_host(S, 100, n=S.size + 1)
    with pytest.raises(ValueError):
        wt.wm_build_host(torch.zeros(4, dtype=torch.int16, device="cuda"), 10)
    h = wt.wm_build_host(np.empty(0, dtype=np.uint16), 10)
    assert h.export().n == 0
    h.free()


def test_wm_build_host_concurrent_streams(wt):
    """Host-memory builds queued on several streams at once (their copies
    share the library's copy stream, their staging buffers the pool) give
    the same structures as device builds, with and without options."""
    import torch
    S = synth.zipf(86, 200003, 65536, 1.1, 2)
    pin = torch.from_numpy(S.view(np.int16)).pin_memory()
    ref = wt.wm_build(pin.to("cuda"), 65536)
    rb, rz = ref.export().bits.copy(), ref.export().zeros.copy()
    ref.free()
    streams = [torch.cuda.Stream() for _ in range(4)]
    opts = [dict(), dict(tau=4), dict(tile_symbols=2048), dict(tau=8, tile_symbols=8192)]
    hs = [wt.wm_build_host(pin, 65536, stream=s, **o) for s, o in zip(streams, opts)]
    for h in hs:
        ex = h.export()
        assert np.array_equal(ex.bits, rb)
        assert np.array_equal(ex.zeros, rz)
        h.free()
