"""The allocation-free directory entry point (rs_dir_build_static).

It serves callers that cannot allocate device memory when they need a
rank/select directory (a component that owns all device memory through its
own manager, a path that must not wait on an allocation, a runtime that
forbids allocation after start-up); its scratch is a static device array
shared by all calls.  The test runs it several times in a row through the C
ABI -- the largest accepted bitvector (exactly 2^30 bits, which fills the
scratch array), then smaller ones and an empty one, so stale scratch from an
earlier call would show -- and compares every directory record and select
sample with the oracle's (exact: integer results, tolerance 0), and the
first two calls also with the regular rs_build entry point.  It sits in its
own file, collected last."""
import numpy as np
import pytest

import oracle
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


def test_static_directory_matches_oracle(wt):
    import torch
    cases = [(1 << 30, 70), ((1 << 24) + 12345, 71), (300001, 72), (0, 73), (2048 * 9 + 1, 74)]
    for call, (nbits, seed) in enumerate(cases):
        words = bitvector(seed, max(nbits, 1))
        d = torch.from_numpy(words.view(np.int64)).to("cuda")
        nsb = (nbits + 2047) // 2048
        cap = nbits // 4096 + 1
        dir_out = torch.full((2 * (nsb + 1),), -1, dtype=torch.int64, device="cuda")
        s0 = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        s1 = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        wt.rs_dir_build_static(d, nbits, dir_out, s0, s1)
        torch.cuda.synchronize()
        got_dir = dir_out.cpu().numpy().view(np.uint64)
        rec = oracle.rank_dir(words, nbits)
        assert np.array_equal(got_dir, rec.reshape(-1)), f"directory, call {call + 1}"
        for b, out in ((0, s0), (1, s1)):
            exp = oracle.select_samples(words, nbits, b)
            got = out.cpu().numpy().view(np.uint64)[:exp.size]
            assert np.array_equal(got, exp), f"select samples of {b}, call {call + 1}"
        if call < 2:
            # the same arrays as the allocating entry point
            h = wt.rs_build(d, nbits)
            ex = h.export()
            assert np.array_equal(got_dir, ex.level_dir(0).reshape(-1))
            h.free()


def test_static_directory_rejects_oversize(wt):
    import torch
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(wt.WaveletError) as ei:
        wt.rs_dir_build_static(dummy, (1 << 30) + 1, dummy, dummy, dummy)
    assert ei.value.status == 6
