"""Seeded synthetic inputs: determinism and distribution sanity."""
import numpy as np

import synth


def test_deterministic_and_chunk_independent():
    a = synth.uniform(5, (1 << 24) + 1000, 256, 1)
    b = synth.uniform(5, (1 << 24) + 1000, 256, 1)
    assert np.array_equal(a, b)
    c = synth.uniform(5, 1000, 256, 1)
    assert np.array_equal(a[:1000], c)  # prefix of chunk 0 does not depend on n
    assert a.max() < 256 and np.abs(np.bincount(a, minlength=256) / a.size - 1 / 256).max() < 1e-3


def test_zipf_shape():
    sigma, s = 4096, 1.1
    z = synth.zipf(7, 1 << 22, sigma, s, 2)
    perm = synth.permutation(7, sigma)
    assert sorted(perm.tolist()) == list(range(sigma))
    h = np.bincount(z.astype(np.int64), minlength=sigma)
    by_rank = h[perm]  # rank r (0-based) is symbol perm[r]
    ratio = by_rank[0] / by_rank[9]
    assert abs(ratio - 10 ** s) / 10 ** s < 0.05
    assert by_rank[0] > by_rank[1] > by_rank[3]


def test_genome():
    g = synth.genome(3, 1 << 20)
    assert g[-1] == 4 and g[:-1].max() <= 3
    assert np.count_nonzero(g == 4) == 1
    runs = np.count_nonzero(np.diff(g[:-1].astype(np.int16)) != 0) + 1
    assert (g.size - 1) / runs > 4.0  # geometric bursts (mean 8) merge into long runs
    cum = synth.markov_table(3)
    assert np.allclose(cum[:, 3], 1.0) and np.all(np.diff(cum, axis=1) >= 0)


def test_batch_plan_cap():
    ln, sig, zf, sd, total = synth.batch_plan(11)
    assert ln.size == 4096 and total == int(ln.sum()) <= (1 << 31)
    assert ln.min() >= 1 << 10 and ln.max() <= 1 << 24
    assert set(np.unique(sig).tolist()) <= {4, 256, 4096, 65536}
    ln2, *_ = synth.batch_plan(11, m=16, cap=1 << 40)
    assert ln2.min() >= 1 << 10 and ln2.max() <= 1 << 24


def test_queries_mix():
    S = synth.uniform(1, 5000, 50, 1)
    op, c, arg = synth.queries(2, S, 50, 30000)
    assert set(np.unique(op).tolist()) == {0, 1, 2}
    assert (arg[op != 2] >= 5000).any() and (c >= 50).any()
