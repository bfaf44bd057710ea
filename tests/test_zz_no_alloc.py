"""The allocation-free directory entry point (rs_dir_build_static).

It serves callers that cannot allocate device memory when they need a
rank/select directory; its scratch is a static device array shared by all
calls.  The test runs it twice in a row through the C ABI -- a large
bitvector, then a smaller one, so stale scratch from the first call would
show -- and compares every directory record and select sample with the
regular rs_build entry point (exact: integer results, tolerance 0).  It sits
in its own file, collected last."""
import numpy as np
import pytest

import synth

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


def bitvector(seed, nbits):
    W = (nbits + 63) // 64
    words = synth.words(seed, W) & synth.words(seed + 1, W)  # about 1/4 ones
    if nbits % 64:
        words[-1] &= np.uint64((1 << (nbits % 64)) - 1)
    return words


def test_static_directory_matches_rs_build(wt):
    import torch
    for call, (nbits, seed) in enumerate([((1 << 24) + 12345, 71), (300001, 72)]):
        words = bitvector(seed, nbits)
        d = torch.from_numpy(words.view(np.int64)).to("cuda")
        nsb = (nbits + 2047) // 2048
        cap = nbits // 4096 + 1
        dir_out = torch.full((2 * (nsb + 1),), -1, dtype=torch.int64, device="cuda")
        s0 = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        s1 = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        wt.rs_dir_build_static(d, nbits, dir_out, s0, s1)
        torch.cuda.synchronize()
        h = wt.rs_build(d, nbits)
        ex = h.export()
        got_dir = dir_out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got_dir, ex.level_dir(0).reshape(-1)), f"directory, call {call + 1}"
        for b, out in ((0, s0), (1, s1)):
            exp = ex.samples(0, b)
            got = out.cpu().numpy().view(np.uint64)[:exp.size]
            assert np.array_equal(got, exp), f"select samples of {b}, call {call + 1}"
        h.free()


def test_static_directory_rejects_oversize(wt):
    import torch
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(wt.WaveletError) as ei:
        wt.rs_dir_build_static(dummy, (1 << 30) + 1, dummy, dummy, dummy)
    assert ei.value.status == 6
