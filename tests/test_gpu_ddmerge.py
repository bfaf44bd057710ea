"""GPU parity of the domain-decomposition merge (Section 4.2): structures of
consecutive pieces of one sequence, merged, equal the oracle's structure of
the whole sequence bit for bit (levels, zero counts, directories, select
samples) and answer queries like it.  Pieces include empty and one-symbol
ones and uneven sizes."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_binary_dirs, oracle_queries, queries_on, to_dev

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


def _cuts(n, kind, rng):
    if kind == "one":
        return [0, n]
    if kind == "two":
        return [0, n // 3, n]
    if kind == "edges":  # an empty piece, a one-symbol piece, two more
        return [0, 0, 1, n // 2, n // 2 + 4097, n]
    c = np.sort(rng.integers(0, n + 1, 7))
    return [0, *c.tolist(), n]


CASES = [
    ("wm", 5, "two", 100003),
    ("wm", 256, "edges", 150000),
    ("wm", 4096, "many", 200000),
    ("wm", 65536, "many", 262147),
    ("wm", 1, "two", 5000),
    ("wt", 5, "edges", 100003),
    ("wt", 300, "many", 180001),
    ("wt", 65536, "two", 262147),
    ("wm", 77, "one", 70000),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-s{c[1]}-{c[2]}-n{c[3]}")
def test_dd_merge_equals_single_build(wt, case):
    kind, sigma, cuts, n = case
    rng = np.random.default_rng(sigma + n)
    S = synth.zipf(60 + sigma, n, sigma, 1.1, 2) if sigma > 1 else np.zeros(n, np.uint16)
    cut = _cuts(n, cuts, rng)
    fn = wt.wm_build if kind == "wm" else wt.wt_build
    parts = [fn(to_dev(np.ascontiguousarray(S[a:b])), sigma) for a, b in zip(cut[:-1], cut[1:])]
    h = wt.dd_merge(parts)
    ex = h.export()
    if kind == "wm":
        ob, oz = oracle.wm_build(S, sigma)
        assert np.array_equal(ex.zeros, oz)
    else:
        ob = oracle.wt_build(S, sigma)
    assert ex.levels == ob.shape[0] and ex.n == n
    assert np.array_equal(ex.bits.reshape(ob.shape), ob)
    check_binary_dirs(ex, list(ob), [n] * ob.shape[0])
    op, c, x = synth.queries(70 + sigma, S, sigma, 20000)
    assert np.array_equal(queries_on(h, S, sigma, op, c, x), oracle_queries(S, sigma, op, c, x))
    for p in parts:
        p.free()
    h.free()


def test_dd_merge_constant_time_select(wt):
    n, sigma = 300001, 1000
    S = synth.zipf(91, n, sigma, 1.1, 2)
    parts = [wt.wm_build(to_dev(np.ascontiguousarray(S[a:b])), sigma)
             for a, b in ((0, 100000), (100000, 100001), (100001, n))]
    h = wt.dd_merge(parts, flags=wt.FLAG_SELECT_O1)
    ex = h.export()
    for l in range(ex.levels):
        for b in (0, 1):
            got = h.export_select(l, b)
            exp = oracle.clark(ex.level(l), n, b)
            for g, e in zip(got, exp):
                assert np.array_equal(g, e)
    op, c, x = synth.queries(92, S, sigma, 20000)
    sel = op == 2
    assert np.array_equal(queries_on(h, S, sigma, op[sel], c[sel], x[sel]),
                          oracle_queries(S, sigma, op[sel], c[sel], x[sel]))
    for p in parts:
        p.free()
    h.free()


def test_dd_merge_rejects_mismatched_parts(wt):
    S = synth.uniform(93, 10000, 300, 2)
    a = wt.wm_build(to_dev(S[:5000].copy()), 300)
    b = wt.wm_build(to_dev(S[5000:].copy()), 301)    # other sigma, same levels
    c = wt.wt_build(to_dev(S[5000:].copy()), 300)    # other kind
    d = wt.wm_build(to_dev(S[5000:].copy()), 300, flags=wt.FLAG_NO_DIRECTORY)
    for bad in ([a, b], [a, c], [a, d], []):
        with pytest.raises(wt.WaveletError) as ei:
            wt.dd_merge(bad)
        assert ei.value.status == 1
    for x in (a, b, c, d):
        x.free()
