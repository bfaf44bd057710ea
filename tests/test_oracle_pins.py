"""Pins of the CPU oracle to things other than itself.

Each check is chosen so that a plausible slip in the oracle (a wrong bit
index, zeros/ones swapped, a partition that ignores node boundaries, an
off-by-one in a directory boundary, a wrong tie-break) fails at least one of
them:

* hand-derived worked examples (Fig. 1 and Fig. 2 inputs, ``tests/golden``);
* closed forms through a library routine: level l of the balanced tree is
  bit L-1-l of ``sorted(S, key=top l bits)`` (Python's sort is stable), and
  level l of the wavelet matrix is the same over the key "top l bits read
  backwards" (the reversed-digit identity of Section 4.3);
* exhaustive enumeration of all sequences with n <= 6 over sigma <= 4;
* brute-force counting (numpy cumulative sums) for rank directories,
  select samples and per-digit directories;
* textbook facts for Huffman codes (Kraft equality, optimal cost from a
  weight-only merge, prefix-freeness, canonical order) and an independent
  dynamic program for length-limited codes.
"""
import heapq
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bitlist(level, nbits):
    return [(int(level[i >> 6]) >> (i & 63)) & 1 for i in range(nbits)]


def L_of(sigma):
    L = 0
    while (1 << L) < sigma:
        L += 1
    return max(L, 1)


def rev(v, nb):
    r = 0
    for _ in range(nb):
        r = (r << 1) | (v & 1)
        v >>= 1
    return r


def wt_closed_form(S, sigma):
    L = L_of(sigma)
    out = []
    for l in range(L):
        T = sorted(S, key=lambda x: x >> (L - l))
        out.append([(x >> (L - 1 - l)) & 1 for x in T])
    return out


def wm_closed_form(S, sigma):
    L = L_of(sigma)
    out = []
    for l in range(L):
        T = sorted(S, key=lambda x: rev(x >> (L - l), l))
        out.append([(x >> (L - 1 - l)) & 1 for x in T])
    return out


def read_golden(name):
    d = {"wt": {}, "wm": {}}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "input":
                d["S"] = [ord(ch) - ord("a") for ch in parts[1]]
            elif parts[0] == "sigma":
                d["sigma"] = int(parts[1])
            elif parts[0] == "wt":
                d["wt"][int(parts[1])] = parts[2]
            elif parts[0] == "wm":
                d["wm"][int(parts[1])] = (parts[2], int(parts[3]))
    return d


@pytest.mark.parametrize("name", ["fig1_cafgaehbhfd.txt", "fig2_abcdefghijklmnop.txt"])
def test_worked_examples(name):
    g = read_golden(name)
    S, sigma = np.array(g["S"], dtype=np.uint32), g["sigma"]
    n = S.size
    wt = oracle.wt_build(S, sigma)
    for l, s in g["wt"].items():
        assert oracle.bits_to_str(wt[l], n) == s
    wm, z = oracle.wm_build(S, sigma)
    for l, (s, zl) in g["wm"].items():
        assert oracle.bits_to_str(wm[l], n) == s
        assert int(z[l]) == zl


def test_exhaustive_small():
    for sigma in (1, 2, 3, 4):
        for n in range(0, 7):
            for S in itertools.product(range(sigma), repeat=n):
                S = list(S)
                a = np.array(S, dtype=np.uint32)
                wt = oracle.wt_build(a, sigma)
                wm, z = oracle.wm_build(a, sigma)
                cf_wt, cf_wm = wt_closed_form(S, sigma), wm_closed_form(S, sigma)
                for l in range(L_of(sigma)):
                    assert bitlist(wt[l], n) == cf_wt[l]
                    assert bitlist(wm[l], n) == cf_wm[l]
                    assert int(z[l]) == cf_wm[l].count(0)


@pytest.mark.parametrize("n,sigma,seed", [(1, 1, 1), (5, 2, 2), (100, 5, 3), (700, 7, 4),
                                         (2500, 256, 5), (3001, 300, 6), (4096, 1000, 7),
                                         (513, 65536, 8)])
def test_closed_forms_random(n, sigma, seed):
    S = synth.uniform(seed, n, sigma, 4)
    Sl = [int(x) for x in S]
    wt = oracle.wt_build(S, sigma)
    wm, z = oracle.wm_build(S, sigma)
    cf_wt, cf_wm = wt_closed_form(Sl, sigma), wm_closed_form(Sl, sigma)
    L = L_of(sigma)
    for l in range(L):
        assert bitlist(wt[l], n) == cf_wt[l], ("wt", l)
        assert bitlist(wm[l], n) == cf_wm[l], ("wm", l)
        assert int(z[l]) == cf_wm[l].count(0)
        # padding beyond n is zero
        W = wt.shape[1]
        assert W % 32 == 0 and W * 64 >= n
        tail = [(int(wt[l][i >> 6]) >> (i & 63)) & 1 for i in range(n, W * 64)]
        assert not any(tail)
    # invariants between the two structures
    assert bitlist(wt[0], n) == bitlist(wm[0], n)
    if L > 1:
        assert bitlist(wt[1], n) == bitlist(wm[1], n)
    for l in range(L):
        ones = sum((x >> (L - 1 - l)) & 1 for x in Sl)
        assert sum(bitlist(wt[l], n)) == ones == n - int(z[l])


def brute_zeros_prefix(level, nbits):
    bits = np.array(bitlist(level, nbits), dtype=np.int64)
    return np.concatenate([[0], np.cumsum(1 - bits)])


@pytest.mark.parametrize("nbits,seed", [(0, 1), (1, 2), (63, 3), (64, 4), (511, 5), (512, 6),
                                        (2047, 7), (2048, 8), (2049, 9), (10000, 10),
                                        (65536 + 77, 11)])
def test_rank_dir_and_select_brute(nbits, seed):
    W = oracle.level_words(nbits)
    words = synth.words(seed, max(W, 1))[:W].copy()
    if nbits % 64:
        words[nbits // 64] &= np.uint64((1 << (nbits % 64)) - 1)
    words[(nbits + 63) // 64:] = 0
    if seed % 3 == 0:  # a sparse variant
        words &= synth.words(seed + 100, max(W, 1))[:W] & synth.words(seed + 200, max(W, 1))[:W]
    Z = brute_zeros_prefix(words, nbits)
    rec = oracle.rank_dir(words, nbits)
    nsb = (nbits + 2047) // 2048
    assert rec.shape == (nsb + 1, 2)
    for s in range(nsb):
        base = 2048 * s
        assert int(rec[s, 0]) == Z[base]
        for b in range(4):
            e = min(base + 512 * b, nbits)
            assert (int(rec[s, 1]) >> (16 * b)) & 0xFFFF == Z[e] - Z[base]
    assert int(rec[nsb, 0]) == Z[nbits] and int(rec[nsb, 1]) == 0
    bl = bitlist(words, nbits)
    for b in (0, 1):
        samp = oracle.select_samples(words, nbits, b)
        cnt = bl.count(b)
        assert samp.size == (cnt + 4095) // 4096
        occ = [p for p, v in enumerate(bl) if v == b]
        for k, p in enumerate(samp):
            assert int(p) == occ[4096 * k]


def huffman_cost(weights):
    h = [w for w in weights if w > 0]
    if len(h) <= 1:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def check_code(hist, ln, code):
    present = [s for s in range(len(hist)) if hist[s] > 0]
    assert all(ln[s] == 0 for s in range(len(hist)) if hist[s] == 0)
    if len(present) >= 2:
        kraft = sum(2.0 ** -int(ln[s]) for s in present)
        assert abs(kraft - 1.0) < 1e-12
    words = {s: format(int(code[s]), "0%db" % int(ln[s])) for s in present}
    # prefix-free
    ws = sorted(words.values())
    for a, b in zip(ws, ws[1:]):
        assert not b.startswith(a)
    # canonical: taken in (len, symbol) order, the codeword intervals
    # [code/2^len, (code+1)/2^len) start at 0 and tile [0, 1) left to right
    order = sorted(present, key=lambda s: (int(ln[s]), s))
    M = max(int(ln[s]) for s in present)
    pos = 0
    for s in order:
        lo = int(code[s]) << (M - int(ln[s]))
        assert lo == pos
        pos = lo + (1 << (M - int(ln[s])))
    if len(present) >= 2:
        assert pos == 1 << M


@pytest.mark.parametrize("seed,sigma,n", [(1, 2, 10), (2, 5, 100), (3, 64, 5000),
                                          (4, 1000, 20000), (5, 300, 300)])
def test_huffman_lengths(seed, sigma, n):
    S = synth.zipf(seed, n, sigma, 1.0, 4)
    hist = np.bincount(S.astype(np.int64), minlength=sigma).astype(np.uint64)
    ln, mx = oracle.huffman_lengths(hist)
    code = oracle.canonical_codes(ln)
    check_code(hist, ln, code)
    assert int((hist * ln.astype(np.uint64)).sum()) == huffman_cost([int(h) for h in hist])
    assert mx == int(ln.max())


def test_huffman_single_and_empty():
    hist = np.zeros(10, dtype=np.uint64)
    ln, mx = oracle.huffman_lengths(hist)
    assert mx == 0 and not ln.any()
    hist[7] = 5
    ln, mx = oracle.huffman_lengths(hist)
    assert mx == 1 and ln[7] == 1 and ln.sum() == 1


def limited_cost_dp(weights, cap):
    """Optimal length-limited prefix-code cost by dynamic programming over
    depths: at each depth some of the available nodes become leaves (the
    heaviest remaining symbols), the others split in two."""
    w = sorted(weights, reverse=True)
    m = len(w)
    suffix = [0] * (m + 1)
    for i in range(m - 1, -1, -1):
        suffix[i] = suffix[i + 1] + w[i]
    from functools import lru_cache

    @lru_cache(maxsize=None)
    def best(d, i, a):
        # d = depth of the available nodes, i = symbols placed, a = available nodes
        if i == m:
            return 0
        if d > cap or a == 0:
            return float("inf")
        res = float("inf")
        for k in range(0, min(a, m - i) + 1):
            rest = a - k
            if i + k == m:
                res = min(res, 0)
                break
            nxt = min(2 * rest, m - i - k)
            res = min(res, suffix[i + k] + best(d + 1, i + k, nxt))
        return res

    return suffix[0] + best(1, 0, 2)


def test_huffman_length_limited_fibonacci():
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    hist = np.array(fib, dtype=np.uint64)
    ln_free, mx_free = oracle.huffman_lengths(hist, cap=64)
    assert mx_free == 39  # Fibonacci weights give the deepest Huffman tree
    for cap in (32, 20, 8, 6):
        ln, mx = oracle.huffman_lengths(hist, cap=cap)
        assert mx <= cap
        code = oracle.canonical_codes(ln)
        check_code(hist, ln, code)
        assert int((hist * ln.astype(np.uint64)).sum()) == limited_cost_dp(fib, cap)


def test_huff_wt_against_definition():
    for seed, sigma, n in [(1, 40, 3000), (2, 5, 777), (3, 2, 100), (4, 300, 5000)]:
        S = synth.zipf(seed, n, sigma, 1.0, 4)
        hist = np.bincount(S.astype(np.int64), minlength=sigma).astype(np.uint64)
        ln, mx = oracle.huffman_lengths(hist)
        code = oracle.canonical_codes(ln)
        bits, woff, nl = oracle.huff_wt_build(S, ln, code)
        cw = [format(int(code[x]), "0%db" % int(ln[x])) for x in S]
        for l in range(mx):
            idx = [i for i in range(n) if len(cw[i]) > l]
            T = sorted(idx, key=lambda i: cw[i][:l])
            exp = [int(cw[i][l]) for i in T]
            assert int(nl[l]) == len(exp)
            got = bitlist(bits[int(woff[l]):int(woff[l + 1])], len(exp))
            assert got == exp
        assert int(nl.sum()) == int((hist * ln.astype(np.uint64)).sum())


@pytest.mark.parametrize("n,sigma,seed", [(1, 5, 1), (1000, 5, 2), (3000, 16, 3),
                                         (2049, 8, 4), (1500, 200, 5), (700, 2, 6)])
def test_mwt_against_binary(n, sigma, seed):
    S = synth.uniform(seed, n, sigma, 4)
    Sl = [int(x) for x in S]
    L = L_of(sigma)
    dig = oracle.mwt_build(S, sigma)
    wt = oracle.wt_build(S, sigma)
    for beta in range((L + 1) // 2):
        l = 2 * beta
        T = sorted(Sl, key=lambda x: x >> (L - l))
        if l + 1 < L:
            exp = [(((x >> (L - 1 - l)) & 1) << 1) | ((x >> (L - 2 - l)) & 1) for x in T]
        else:
            exp = [(x >> (L - 1 - l)) & 1 for x in T]
        got = [(int(dig[beta][i >> 5]) >> (2 * (i & 31))) & 3 for i in range(n)]
        assert got == exp
        # high bit plane equals the binary level 2*beta bitmap
        hi = [(d >> 1) if l + 1 < L else d for d in got]
        assert hi == bitlist(wt[l], n)
        rec = oracle.mwt_dir(dig[beta], n)
        cum = np.zeros((n + 1, 4), dtype=np.int64)
        for i, d in enumerate(got):
            cum[i + 1] = cum[i]
            cum[i + 1, d] += 1
        nsb = (n + 1023) // 1024
        for s in range(nsb):
            for v in range(4):
                assert int(rec[s, v]) == cum[1024 * s, v]
            for b in range(4):
                e = min(1024 * s + 256 * b, n)
                for v in range(4):
                    assert (int(rec[s, 4 + b]) >> (16 * v)) & 0xFFFF == cum[e, v] - cum[1024 * s, v]
        for v in range(4):
            assert int(rec[nsb, v]) == cum[n, v]


def test_queries_definition():
    S = synth.zipf(9, 600, 20, 1.1, 4)
    Sl = [int(x) for x in S]
    n, sigma = len(Sl), 20
    i = np.arange(0, n + 3, dtype=np.uint64)
    acc = oracle.access(S, i)
    for t, v in enumerate(i):
        assert int(acc[t]) == (Sl[int(v)] if v < n else 2 ** 64 - 1)
    cs = np.repeat(np.arange(0, sigma + 1, dtype=np.uint32), 7)
    ii = np.tile(np.array([0, 1, 50, 299, 598, 599, 600], dtype=np.uint64), sigma + 1)
    rk = oracle.rank(S, sigma, cs, ii)
    for t in range(cs.size):
        c, x = int(cs[t]), int(ii[t])
        exp = sum(1 for j in range(x + 1) if Sl[j] == c) if (x < n and c < sigma) else 2 ** 64 - 1
        assert int(rk[t]) == exp
    kk = np.tile(np.array([0, 1, 2, 5, 40, 1000], dtype=np.uint64), sigma + 1)
    cs2 = np.repeat(np.arange(0, sigma + 1, dtype=np.uint32), 6)
    sl = oracle.select(S, sigma, cs2, kk)
    for t in range(cs2.size):
        c, k = int(cs2[t]), int(kk[t])
        occ = [j for j in range(n) if Sl[j] == c] if c < sigma else []
        exp = occ[k - 1] if (c < sigma and 1 <= k <= len(occ)) else 2 ** 64 - 1
        assert int(sl[t]) == exp


# ---------------------------------------------------------------------------
# constant-time select directory (§5.1 select after Clark): answers read
# from the oracle's arrays by the definition in oracle.h equal the brute-force
# position of every occurrence; small thresholds make all three kinds of
# range and sub-range appear
# ---------------------------------------------------------------------------
def _clark_answer(desc, sub, sparse, huge, samp, bits, nbits, b, j, width=1):
    k = j >> 12
    d = int(desc[k])
    if d >> 63:
        return int(huge[(d & ((1 << 63) - 1)) + (j & 4095)])
    i = (j >> 8) & 15
    mask = (d >> 40) & 0xFFFF
    S1 = int(samp[k])
    if (mask >> i) & 1:
        s = (d & ((1 << 40) - 1)) + bin(mask & ((1 << i) - 1)).count("1")
        return S1 + int(sparse[256 * s + (j & 255)])
    p = S1 + int(sub[16 * k + i])
    need = j & 255  # occurrences to skip after the sub-range's first one
    while True:
        q = p * width
        if ((int(bits[q >> 6]) >> (q & 63)) & ((1 << width) - 1)) == b:
            if need == 0:
                return p
            need -= 1
        p += 1


@pytest.mark.parametrize("seed,nbits,density,huge_min,sparse_min", [
    (1, 30000, 0.5, 1 << 32, 1 << 16),
    (2, 200000, 0.02, 1 << 14, 1 << 11),
    (3, 200000, 0.002, 1 << 14, 1 << 11),
    (4, 120000, 0.98, 1 << 13, 1 << 10),
    (5, 65536, 0.0001, 1 << 12, 1 << 9),
    (6, 5000, 0.3, 1 << 32, 1 << 16),
])
def test_clark_select_answers_every_occurrence(seed, nbits, density, huge_min, sparse_min):
    rng = np.random.default_rng(seed)
    # runs of dense and sparse stretches, so ranges of every kind appear
    raw = rng.random(nbits)
    dens = np.where((np.arange(nbits) // 7000) % 3 == 0, density, min(0.5, density * 50))
    x = (raw < dens).astype(np.uint8)
    words = np.zeros(oracle.level_words(nbits), dtype=np.uint64)
    packed = np.packbits(x, bitorder="little")
    words.view(np.uint8)[:packed.size] = packed
    kinds = set()
    for b in (0, 1):
        pos = np.nonzero(x == b)[0]
        desc, sub, sparse, huge = oracle.clark(words, nbits, b, huge_min, sparse_min)
        samp = oracle.select_samples(words, nbits, b)
        assert desc.size == (pos.size + 4095) // 4096 == samp.size
        for k in range(desc.size):
            d = int(desc[k])
            kinds.add("huge" if d >> 63 else ("sparse" if (d >> 40) & 0xFFFF else "dense"))
            if not d >> 63:
                assert sub[16 * k] == 0
        # every occurrence on small inputs; every 4096-th, every sub-range
        # start and a seeded sample on the larger ones
        js = np.arange(pos.size)
        if pos.size > 20000:
            js = np.unique(np.concatenate([js[::256], js[255::256], js[-300:],
                                           rng.integers(0, pos.size, 6000)]))
        for j in js:
            j = int(j)
            assert _clark_answer(desc, sub, sparse, huge, samp, words, nbits, b, j) == pos[j], (b, j)
    if seed in (2, 3, 5):
        assert "huge" in kinds or "sparse" in kinds


# ---------------------------------------------------------------------------
# generalized select on 4-ary digit levels (§5.2, select per character): the
# same sampled and constant-time structures over the occurrences of each
# digit value; brute force over the digit array
# ---------------------------------------------------------------------------
def _digit_words(x):
    n = x.size
    words = np.zeros(oracle.level_words(2 * n), dtype=np.uint64)
    for v in range(4):
        pos = np.nonzero(x == v)[0].astype(np.uint64) * np.uint64(2)
        if v & 1:
            np.bitwise_or.at(words, (pos >> np.uint64(6)).astype(np.int64),
                             np.left_shift(np.uint64(1), pos & np.uint64(63)))
        if v & 2:
            q = pos + np.uint64(1)
            np.bitwise_or.at(words, (q >> np.uint64(6)).astype(np.int64),
                             np.left_shift(np.uint64(1), q & np.uint64(63)))
    return words


@pytest.mark.parametrize("seed,n,probs,huge_min,sparse_min", [
    (1, 30000, (0.25, 0.25, 0.25, 0.25), 1 << 32, 1 << 16),
    (2, 150000, (0.97, 0.01, 0.01, 0.01), 1 << 14, 1 << 11),
    (3, 150000, (0.5, 0.499, 0.0005, 0.0005), 1 << 13, 1 << 10),
    (4, 70000, (0.1, 0.2, 0.3, 0.4), 1 << 12, 1 << 9),
    (5, 5000, (0.0, 1.0, 0.0, 0.0), 1 << 32, 1 << 16),
])
def test_digit_select_structures_answer_every_occurrence(seed, n, probs, huge_min, sparse_min):
    rng = np.random.default_rng(100 + seed)
    x = rng.choice(4, size=n, p=probs).astype(np.uint8)
    # stretches where value 0 takes over, so long ranges appear for the others
    x[(np.arange(n) // 9000) % 4 == 1] = 0
    words = _digit_words(x)
    # the packing itself against the oracle's 4-ary levels of a sigma-4 text
    assert np.array_equal(words, oracle.mwt_build(x.astype(np.uint32), 4)[0])
    kinds = set()
    for d in range(4):
        pos = np.nonzero(x == d)[0]
        samp = oracle.digit_samples(words, n, d)
        assert np.array_equal(samp, pos[::4096].astype(np.uint64))
        desc, sub, sparse, huge = oracle.clark_digits(words, n, d, huge_min, sparse_min)
        assert desc.size == (pos.size + 4095) // 4096
        for k in range(desc.size):
            dk = int(desc[k])
            kinds.add("huge" if dk >> 63 else ("sparse" if (dk >> 40) & 0xFFFF else "dense"))
        js = np.arange(pos.size)
        if pos.size > 20000:
            js = np.unique(np.concatenate([js[::256], js[255::256], js[-300:],
                                           rng.integers(0, pos.size, 5000)]))
        for j in js:
            j = int(j)
            got = _clark_answer(desc, sub, sparse, huge, samp, words, n, d, j, width=2)
            assert got == pos[j], (d, j)
    if seed in (2, 3, 4):
        assert {"huge", "sparse"} & kinds
