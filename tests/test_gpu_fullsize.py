"""Parity with the oracle, bit-exact, at 2^25 symbols: 8192 tiles, so the
per-tile prefix tables span many 256-tile chunks and the chunk prefixes
carry counts across them (single builds and a batch of four sequences).
The workloads at their full sizes are compared in test_gpu_configs.py."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_binary_dirs, to_dev

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


@pytest.mark.parametrize("kind,tile", [("wm", 0), ("wt", 0), ("wm", 2048), ("wm", 8192)])
def test_parity_across_prefix_chunks(wt, kind, tile):
    n, sigma = 1 << 25, 4096
    S = synth.zipf(77, n, sigma, 1.1, 2)
    if kind == "wm":
        h = wt.wm_build(to_dev(S), sigma, tile_symbols=tile)
    else:
        h = wt.wt_build(to_dev(S), sigma)
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
