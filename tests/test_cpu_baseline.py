"""The multi-threaded CPU comparison build (cpu_baseline/) against the
oracle: levels, zero counts, rank records and select samples, bit-exact, for
several thread counts (chunk boundaries fall inside and between words)."""
import numpy as np
import pytest

import cpu_baseline
import oracle
import synth


@pytest.mark.parametrize("n,sigma,threads", [(1, 2, 3), (63, 5, 2), (4097, 77, 5),
                                             (100003, 300, 7), (1 << 20, 1 << 16, 16)])
def test_cpu_parallel_wm_equals_oracle(n, sigma, threads):
    S = synth.zipf(n % 97 + 3, n, sigma, 1.1, 2)
    L = oracle.levels(sigma)
    bits, zeros, dirs, samp = cpu_baseline.wm_build(S, L, threads)
    ob, oz = oracle.wm_build(S, sigma)
    assert np.array_equal(bits, ob) and np.array_equal(zeros, oz)
    for l in range(L):
        assert np.array_equal(dirs[l], oracle.rank_dir(ob[l], n).reshape(-1, 2)), l
        for b in (0, 1):
            s = oracle.select_samples(ob[l], n, b)
            assert np.array_equal(samp[l, b, :s.size], s), (l, b)
