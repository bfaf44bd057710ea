"""GPU parity of the batched build, the multi-structure query launch, the
autotuner and the serving loop, against the CPU oracle (all integer: every
word, record, sample, zero count and answer bit-exact).

The batched workload follows the batched configuration's recipe (lengths
log-uniform, sigma from {4, 256, 4096, 65536}, uniform or Zipf(1.1) by coin
flip, uint16), at sizes the oracle finishes in seconds, plus edge sequences
(empty, one symbol, sigma 1 and 2, 8- and 32-bit symbols, a 2^20 alphabet)."""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import UMAX, check_binary_dirs, from_dev_u64, oracle_queries, queries_on, to_dev

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


def batch_inputs(seed, m, lo, hi, cap=1 << 31):
    ln, sig, zf, sd, _ = synth.batch_plan(seed, m, lo, hi, cap)
    seqs = []
    for i in range(m):
        n, s = int(ln[i]), int(sig[i])
        if zf[i]:
            S = synth.zipf(int(sd[i]), n, s, 1.1, 2)
        else:
            S = synth.uniform(int(sd[i]), n, s, 2)
        seqs.append((S, s))
    return seqs


EDGE = [
    (np.zeros(0, np.uint16), 7),
    (np.array([3], np.uint16), 4),
    (np.zeros(5000, np.uint16), 1),
    (synth.uniform(91, 9000, 2, 2), 2),
    (synth.uniform(92, 4096, 256, 1), 256),          # 8-bit symbols, one full tile
    (synth.uniform(93, 12289, 1 << 20, 4), 1 << 20),  # 32-bit working elements
    (synth.zipf(94, 70001, 65536, 1.1, 2), 65536),
    (synth.uniform(95, 4097, 3, 2), 3),
]


def check_wm(ex, S, sigma):
    ob, oz = oracle.wm_build(S, sigma)
    assert ex.levels == ob.shape[0]
    assert np.array_equal(ex.bits.reshape(ob.shape), ob)
    assert np.array_equal(ex.zeros, oz)
    check_binary_dirs(ex, list(ob), [S.size] * ob.shape[0])


@pytest.mark.parametrize("tau", [0, 3, 8])
def test_batch_parity(wt, tau):
    seqs = batch_inputs(7 + tau, 40, 10, 16) + EDGE
    dev = [to_dev(S) for S, _ in seqs]
    hs = wt.wm_batch_build(dev, [s for _, s in seqs], ns=[S.size for S, _ in seqs], tau=tau)
    assert len(hs) == len(seqs)
    for (S, sigma), h in zip(seqs, hs):
        check_wm(h.export(), S, sigma)
    # freeing in any order keeps the others valid (shared allocation)
    for h in hs[::2]:
        h.free()
    for (S, sigma), h in list(zip(seqs, hs))[1::2][:4]:
        check_wm(h.export(), S, sigma)
    for h in hs[1::2]:
        h.free()


def test_batch_queries_match_oracle(wt):
    seqs = batch_inputs(21, 12, 10, 15)
    dev = [to_dev(S) for S, _ in seqs]
    hs = wt.wm_batch_build(dev, [s for _, s in seqs])
    for i, ((S, sigma), h) in enumerate(zip(seqs, hs)):
        op, c, x = synth.queries(100 + i, S, sigma, 3000)
        got = queries_on(h, S, sigma, op, c, x)
        assert np.array_equal(got, oracle_queries(S, sigma, op, c, x))


def test_batch_symbol_error_is_per_sequence(wt):
    good = synth.uniform(31, 10000, 16, 2)
    bad = synth.uniform(32, 10000, 16, 2)
    bad[777] = 16
    hs = wt.wm_batch_build([to_dev(good), to_dev(bad), to_dev(good)], [16, 16, 16])
    hs[0].sync()
    hs[2].sync()
    with pytest.raises(wt.WaveletError) as e:
        hs[1].sync()
    assert e.value.status == 2
    check_wm(hs[2].export(), good, 16)


def test_batch_empty_and_invalid(wt):
    assert wt.wm_batch_build([], []) == []
    with pytest.raises(wt.WaveletError):
        wt.wm_batch_build([to_dev(synth.uniform(1, 10, 4, 2))], [0])


def test_query_multi(wt):
    rng = np.random.Generator(np.random.PCG64(5))
    a = synth.zipf(41, 30000, 1000, 1.1, 2)
    b = synth.uniform(42, 20000, 5, 1)
    c_ = synth.uniform(43, 25000, 300, 2)
    hs = [wt.wm_build(to_dev(a), 1000), wt.wt_build(to_dev(b), 5),
          wt.huff_wt_build(to_dev(c_), 300), wt.multiary_build(to_dev(a), 1000)]
    data = [(a, 1000), (b, 5), (c_, 300), (a, 1000)]
    q = 20000
    sid = rng.integers(0, 5, size=q).astype(np.uint32)  # 4 = out of range
    op = np.zeros(q, np.uint8)
    cc = np.zeros(q, np.uint32)
    xx = np.zeros(q, np.uint64)
    exp = np.full(q, UMAX, dtype=np.uint64)
    for s in range(4):
        m = sid == s
        S, sg = data[s]
        o, c2, x2 = synth.queries(200 + s, S, sg, int(m.sum()))
        op[m], cc[m], xx[m] = o, c2, x2
        exp[m] = oracle_queries(S, sg, o, c2, x2)
    bad_op = rng.random(q) < 0.01
    op[bad_op] = 3
    exp[bad_op] = UMAX
    import torch
    out = torch.empty(q, dtype=torch.int64, device="cuda")
    wt.query_multi(hs, to_dev(sid), to_dev(op), to_dev(cc), to_dev(xx), out)
    assert np.array_equal(from_dev_u64(out), exp)


def test_autotune(wt):
    S = synth.zipf(51, 1 << 20, 4096, 1.1, 2)
    d = to_dev(S)
    try:
        best, ms = wt.wm_autotune(d, 4096)
        assert 1 <= best <= 8
        assert all(v > 0 for v in ms[:8])
        # builds with tau = 0 now use the tuned value; the result is tau-invariant
        h = wt.wm_build(d, 4096)
        check_wm(h.export(), S, 4096)
        hs = wt.wm_batch_build([d], [4096])
        check_wm(hs[0].export(), S, 4096)
    finally:
        wt.wm_autotune_clear()


def test_batch_object(wt):
    """One object for a whole batched build: its structures equal the
    oracle's, answer queries, report per-sequence statuses (a symbol >= sigma
    in one sequence fails that one only), and are released together."""
    seqs = [(synth.zipf(90 + i, n, s, 1.1, 2), s) for i, (n, s) in
            enumerate([(50001, 4096), (7, 4), (300000, 65536), (0, 256), (8192, 2)])]
    bad = synth.uniform(99, 5000, 300, 2)
    bad[17] = 299
    ds = [to_dev(S) for S, _ in seqs] + [to_dev(bad)]
    b = wt.wm_batch_build_one(ds, [s for _, s in seqs] + [200])
    assert len(b) == 6
    st = b.sync()
    assert list(st[:5]) == [0] * 5 and st[5] == 2
    for i, (S, sigma) in enumerate(seqs):
        h = b.handle(i)
        check_wm(h.export(), S, sigma)
        if S.size:
            q = 1000
            op, c, arg = synth.queries(100 + i, S, sigma, q)
            assert np.array_equal(queries_on(h, S, sigma, op, c, arg),
                                  oracle_queries(S, sigma, op, c, arg))
        h.free()  # a member's free only drops the view
    b.free()
    b.free()


def test_autotune_config(wt):
    """The whole-configuration tuner: (tau, tile size, CTAs per SM) and K;
    builds with zero options then take the recorded triple (wm_tuning reports
    it), and the result does not depend on it."""
    n = (1 << 20) + 4097
    S = synth.zipf(52, n, 65536, 1.1, 2)
    d = to_dev(S)
    try:
        t = wt.wm_autotune_config(d, 65536)
        assert 1 <= t["tau"] <= 8 and t["tile_symbols"] in (2048, 4096, 8192)
        assert t["ctas_per_sm"] in (0, 3, 4) and t["ms"] > 0
        assert t["k_chunks"] == (n + t["tile_symbols"] - 1) // t["tile_symbols"]
        u = wt.wm_tuning(n, 65536)
        assert (u["tau"], u["tile_symbols"], u["ctas_per_sm"], u["k_chunks"]) == \
            (t["tau"], t["tile_symbols"], t["ctas_per_sm"], t["k_chunks"])
        h = wt.wm_build(d, 65536)
        check_wm(h.export(), S, 65536)
        h.free()
    finally:
        wt.wm_autotune_clear()
    assert wt.wm_tuning(n, 65536)["tile_symbols"] == 4096


def _alone_answers(wt, seqs, qs):
    """Each request on its own: one plain build per sequence, one query call
    per op and structure.  qs hold sequence indices (-1: no structure)."""
    hs = [wt.wm_build(to_dev(S), s) for S, s in seqs]
    outs = []
    for k_idx, op, c, x in qs:
        out = np.full(k_idx.size, UMAX, dtype=np.uint64)
        for k in range(len(seqs)):
            m = k_idx == k
            if m.any():
                S, s = seqs[k]
                out[m] = queries_on(hs[k], S, s, op[m], c[m], x[m])
        outs.append(out)
    for h in hs:
        h.free()
    return outs


def test_server_mix_equals_alone(wt):
    seqs = batch_inputs(61, 16, 10, 15)
    srv = wt.Server(budget_bytes=1 << 30)
    try:
        rng = np.random.Generator(np.random.PCG64(9))
        ids, reqs, qs = [], [], []
        for i, (S, s) in enumerate(seqs):
            ids.append(srv.submit_build(S, s))
            if i % 3 == 2:
                # queries over the structures submitted so far (some still building)
                q = 5000
                k = rng.integers(0, len(ids), size=q)
                sid = np.array(ids, dtype=np.uint64)[k]
                op = np.zeros(q, np.uint8)
                c = np.zeros(q, np.uint32)
                x = np.zeros(q, np.uint64)
                for j in np.unique(k):
                    m = k == j
                    S2, s2 = seqs[j]
                    op[m], c[m], x[m] = synth.queries(300 + i * 100 + int(j), S2, s2, int(m.sum()))
                reqs.append(srv.submit_queries(sid, op, c, x))
                qs.append((k, op, c, x))
        got = []
        for r, (k, _, _, _) in zip(reqs, qs):
            st, t0, t1, out = srv.poll(r, k.size)
            assert st == 0 and t1 >= t0
            got.append(out)
        for i in ids:
            st, _, _, _ = srv.poll(i)
            assert st == 0
        alone = _alone_answers(wt, seqs, qs)
        for g, a, (k, op, c, x) in zip(got, alone, qs):
            assert np.array_equal(g, a)
            exp = np.zeros(k.size, np.uint64)
            for j in np.unique(k):
                m = k == j
                S2, s2 = seqs[j]
                exp[m] = oracle_queries(S2, s2, op[m], c[m], x[m])
            assert np.array_equal(g, exp)
        # released and unknown structures answer UINT64_MAX
        srv.release(ids[0])
        r = srv.submit_queries(np.array([ids[0], 10 ** 9], np.uint64), np.array([0, 0], np.uint8),
                               np.zeros(2, np.uint32), np.zeros(2, np.uint64))
        st, _, _, out = srv.poll(r, 2)
        assert st == 0 and np.all(out == UMAX)
        st = srv.stats()
        assert st["structures"] == len(seqs) - 1
    finally:
        srv.close()


def test_server_budget_admission(wt):
    seqs = [(synth.uniform(70 + i, 50000, 256, 2), 256) for i in range(6)]
    budget = (16 << 20) + 800_000  # the per-batch overhead and about two builds
    srv = wt.Server(budget_bytes=budget)
    try:
        big = srv.submit_build(synth.uniform(80, 1 << 22, 256, 2), 256)
        st, _, _, _ = srv.poll(big)
        assert st == 3  # needs more than the whole budget
        ids = [srv.submit_build(S, s) for S, s in seqs]
        done = set()
        t_end = time.time() + 60
        while len(done) < len(ids) and time.time() < t_end:
            for i in ids:
                if i in done:
                    continue
                st, _, _, _ = srv.poll(i, wait=False)
                if st is not None:
                    assert st == 0
                    assert srv.stats()["used_bytes"] <= budget
                    done.add(i)
                    srv.release(i)  # gives the memory back for the next ones
            time.sleep(0.01)
        assert len(done) == len(ids)
        assert srv.stats()["build_batches"] >= 3
    finally:
        srv.close()
