"""Shared helpers of the GPU parity tests (device marshalling, comparisons)."""
import numpy as np

import oracle

UMAX = np.uint64(2 ** 64 - 1)
_VIEW = {1: np.uint8, 2: np.int16, 4: np.int32}


def to_dev(a: np.ndarray):
    import torch
    a = np.ascontiguousarray(a)
    v = a.view(_VIEW[a.dtype.itemsize]) if a.dtype.itemsize in (2, 4) else a
    if a.dtype.itemsize == 8:
        v = a.view(np.int64)
    return torch.from_numpy(v).to("cuda")


def from_dev_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def queries_on(h, S, sigma, q_op, q_c, q_arg):
    """Run a mixed query batch through the C ABI, grouped by op."""
    import torch
    out = np.zeros(q_op.size, dtype=np.uint64)
    for op in (0, 1, 2):
        m = q_op == op
        if not m.any():
            continue
        c = to_dev(q_c[m].astype(np.uint32))
        x = to_dev(q_arg[m].astype(np.uint64))
        o = torch.empty(int(m.sum()), dtype=torch.int64, device="cuda")
        if op == 0:
            h.access(x, o)
        elif op == 1:
            h.rank(c, x, o)
        else:
            h.select(c, x, o)
        out[m] = from_dev_u64(o)
    return out


def oracle_queries(S, sigma, q_op, q_c, q_arg):
    out = np.zeros(q_op.size, dtype=np.uint64)
    m = q_op == 0
    out[m] = oracle.access(S, q_arg[m])
    m = q_op == 1
    out[m] = oracle.rank(S, sigma, q_c[m], q_arg[m])
    m = q_op == 2
    out[m] = oracle.select(S, sigma, q_c[m], q_arg[m])
    return out


def check_binary_dirs(ex, bits_by_level, nbits_by_level):
    """Directory records and select samples of every level vs the oracle."""
    for l, (bl, nb) in enumerate(zip(bits_by_level, nbits_by_level)):
        rec = oracle.rank_dir(bl, nb)
        got = ex.level_dir(l)
        assert np.array_equal(got, rec), f"rank directory of level {l}"
        # the level's zero count: the oracle directory's total
        assert int(ex.zeros[l]) == int(rec[-1, 0]), f"zeros of level {l}"
        for b in (0, 1):
            s = oracle.select_samples(bl, nb, b)
            assert np.array_equal(ex.samples(l, b), s), f"select samples level {l} bit {b}"
