"""GPU checks beyond the small parity sizes.

* Parity with the oracle, bit-exact, at 2^25 symbols: 8192 tiles, so the
  per-tile prefix tables span many 256-tile chunks and the chunk prefixes
  carry counts across them.
* The headline workload at full size, in the launch configuration the
  benchmark times (wavelet matrix of n = 2^30 uint16 Zipf(1.1) symbols over
  2^16): properties that hold at any size.  Each level of a wavelet matrix
  or balanced wavelet tree holds every element once, so its number of ones
  equals the number of symbols with that bit set (from the input alone).
  Sampled access / rank / select answers are compared with brute force on
  the host input.
* The batched workload (4096 sequences, 2^31 symbols) with the same checks
  per sequence."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_binary_dirs, from_dev_u64, to_dev

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


@pytest.mark.parametrize("kind", ["wm", "wt"])
def test_parity_across_prefix_chunks(wt, kind):
    n, sigma = 1 << 25, 4096
    S = synth.zipf(77, n, sigma, 1.1, 2)
    fn = wt.wm_build if kind == "wm" else wt.wt_build
    h = fn(to_dev(S), sigma)
    ex = h.export()
    ob = oracle.wm_build(S, sigma)[0] if kind == "wm" else oracle.wt_build(S, sigma)
    assert np.array_equal(ex.bits.reshape(ob.shape), ob)
    check_binary_dirs(ex, list(ob), [n] * ob.shape[0])
    h.free()


def test_batch_parity_across_prefix_chunks(wt):
    seqs = [(synth.uniform(80 + i, n, s, 2), s) for i, (n, s) in
            enumerate([(1 << 23, 256), (3 << 22, 65536), (1 << 22, 4), (5 << 21, 4096)])]
    hs = wt.wm_batch_build([to_dev(S) for S, _ in seqs], [s for _, s in seqs])
    for (S, sigma), h in zip(seqs, hs):
        ob, oz = oracle.wm_build(S, sigma)
        ex = h.export()
        assert np.array_equal(ex.bits.reshape(ob.shape), ob)
        assert np.array_equal(ex.zeros, oz)


def _level_ones(S, L):
    """Ones of each level of a WM / balanced WT: symbols with bit L-1-l set."""
    return np.array([int(np.count_nonzero((S >> (L - 1 - l)) & 1)) for l in range(L)],
                    dtype=np.uint64)


def _dir_totals(ex):
    return np.array([int(ex.level_dir(l)[-1, 0]) for l in range(ex.levels)], dtype=np.uint64)


def _sampled_queries(wt, h, S, sigma, rng, nsym=6, q=3000):
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
        assert np.array_equal(from_dev_u64(out), np.searchsorted(pos, ii, side="right").astype(np.uint64))
        kk = rng.integers(1, pos.size + 1, q).astype(np.uint64)
        h.select(to_dev(cc), to_dev(kk), out)
        assert np.array_equal(from_dev_u64(out), pos[(kk - 1).astype(np.int64)])


def test_headline_workload_full_size(wt):
    import torch
    n, sigma = 1 << 30, 1 << 16
    pin = torch.empty(n, dtype=torch.int16).pin_memory()
    synth.zipf(synth.SEED_BASE + 2, n, sigma, 1.1, 2, addr=pin.data_ptr())
    S = pin.numpy().view(np.uint16)
    d = pin.to("cuda")
    h = wt.wm_build(d, sigma)
    ex = h.export()
    ones = _level_ones(S, 16)
    assert np.array_equal(np.uint64(n) - ex.zeros, ones)
    assert np.array_equal(_dir_totals(ex), ex.zeros)
    del ex
    _sampled_queries(wt, h, S, sigma, np.random.default_rng(5))
    h.free()


def test_batched_workload_full_size(wt):
    import torch
    m = 4096
    ln, sig, zf, sd, total = synth.batch_plan(synth.SEED_BASE + 5, m, 10, 24, 1 << 31)
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
    check = set(rng.choice(m, 24, replace=False).tolist()) | {int(np.argmax(ln))}
    for i, h in enumerate(hs):
        if i not in check:
            continue
        S = host[int(offs[i]):int(offs[i]) + int(ln[i])]
        L = oracle.levels(int(sig[i]))
        ex = h.export()
        assert np.array_equal(np.uint64(S.size) - ex.zeros, _level_ones(S, L))
        assert np.array_equal(_dir_totals(ex), ex.zeros)
        _sampled_queries(wt, h, S, int(sig[i]), rng, nsym=3, q=500)
    for h in hs:
        h.free()
