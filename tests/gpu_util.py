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


_POOL = None


def oracle_pool():
    """Thread pool for oracle calls at full size: the oracle is C behind ctypes,
    which releases the GIL, so its builds and directory scans run in parallel
    on the host cores while the GPU works (threads, never a forked process)."""
    global _POOL
    if _POOL is None:
        import concurrent.futures as cf
        import os
        _POOL = cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 8)
    return _POOL


def _rank_dir_job(got, bl, nb, zeros, l):
    rec = oracle.rank_dir(bl, nb)
    if not np.array_equal(got, rec):
        bad = np.flatnonzero(np.any(got != rec, axis=1))
        return f"rank directory of level {l}: {bad.size} records differ, first {int(bad[0])}"
    if int(zeros) != int(rec[-1, 0]):
        return f"zeros of level {l}"
    return None


def _samples_job(got, fn, dl, nb, v, what):
    if not np.array_equal(got, fn(dl, nb, v)):
        return f"{what}: select samples of value {v}"
    return None


def check_binary_dirs_parallel(ex, bits_by_level, nbits_by_level):
    """check_binary_dirs with every level's oracle scans (directory, samples
    of zeros, samples of ones) spread over the pool."""
    pool = oracle_pool()
    futs = []
    for l, (bl, nb) in enumerate(zip(bits_by_level, nbits_by_level)):
        futs.append(pool.submit(_rank_dir_job, ex.level_dir(l), bl, nb, ex.zeros[l], l))
        for b in (0, 1):
            futs.append(pool.submit(_samples_job, ex.samples(l, b), oracle.select_samples, bl,
                                    nb, b, f"level {l}"))
    errs = [e for e in (f.result() for f in futs) if e]
    assert not errs, errs


def _digit_dir_job(got, dl, nd, b):
    if not np.array_equal(got, oracle.mwt_dir(dl, nd)):
        return f"digit directory of level {b}"
    return None


def check_digit_dirs_parallel(ex, digit_levels, ndig):
    """Per-digit-value directory records and digit samples of every digit
    level of a 4-ary tree against the oracle, spread over the pool."""
    pool = oracle_pool()
    futs = []
    for b, dl in enumerate(digit_levels):
        futs.append(pool.submit(_digit_dir_job, ex.level_dir(b), dl, ndig, b))
        for d in range(4):
            futs.append(pool.submit(_samples_job, ex.samples(b, d), oracle.digit_samples, dl,
                                    ndig, d, f"digit level {b}"))
    errs = [e for e in (f.result() for f in futs) if e]
    assert not errs, errs


def first_diff(a: np.ndarray, b: np.ndarray):
    """(equal, message) for two word arrays: the first differing word, if any."""
    if a.shape != b.shape:
        return False, f"shapes {a.shape} vs {b.shape}"
    if np.array_equal(a, b):
        return True, ""
    i = int(np.flatnonzero(a.reshape(-1) != b.reshape(-1))[0])
    return False, f"word {i}: {int(a.reshape(-1)[i]):#x} vs {int(b.reshape(-1)[i]):#x}"
