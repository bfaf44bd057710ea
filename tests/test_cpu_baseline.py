"""The multi-threaded CPU comparison builds (cpu_baseline/: levelwise
splits, and big levels with table-driven short lists) against the oracle:
levels, zero counts, rank records and select samples, bit-exact, for several
thread counts (chunk boundaries fall inside and between words) and level
counts that are and are not multiples of the short lists' 4 bits."""
import numpy as np
import pytest

import cpu_baseline
import oracle
import synth


@pytest.mark.parametrize("short", [False, True])
@pytest.mark.parametrize("n,sigma,threads", [(1, 2, 3), (63, 5, 2), (4097, 77, 5), (5, 3, 1),
                                             (100003, 300, 7), (65, 1 << 16, 1),
                                             (1 << 20, 1 << 16, 16), (70001, 1 << 13, 3)])
def test_cpu_parallel_wm_equals_oracle(n, sigma, threads, short):
    S = synth.zipf(n % 97 + 3, n, sigma, 1.1, 2)
    L = oracle.levels(sigma)
    bits, zeros, dirs, samp = cpu_baseline.wm_build(S, L, threads, short_lists=short)
    ob, oz = oracle.wm_build(S, sigma)
    assert np.array_equal(bits, ob) and np.array_equal(zeros, oz)
    for l in range(L):
        assert np.array_equal(dirs[l], oracle.rank_dir(ob[l], n).reshape(-1, 2)), l
        for b in (0, 1):
            s = oracle.select_samples(ob[l], n, b)
            assert np.array_equal(samp[l, b, :s.size], s), (l, b)
