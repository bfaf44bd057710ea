"""Seeded synthetic workloads (shared by tests, bench and oracle comparisons).

Holds no wavelet-tree arithmetic: only random draws and the workload
distributions, implemented in ``gen.c`` (xoshiro256** seeded via splitmix64,
generated in independent 2^24-symbol chunks, OpenMP-parallel; the output does
not depend on the thread count).  Every function returns numpy arrays or
fills a caller buffer given by address.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

#: seeds of the five workloads (one per configuration)
SEED_BASE = 0x16100352400

_WIDTH_DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SRC) > os.path.getmtime(_SO):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            c = ctypes
            lib.syn_uniform.argtypes = [c.c_uint64, c.c_uint64, c.c_uint32, c.c_int, c.c_void_p]
            lib.syn_zipf.restype = c.c_int
            lib.syn_zipf.argtypes = [c.c_uint64, c.c_uint64, c.c_uint32, c.c_double, c.c_int,
                                     c.c_void_p]
            lib.syn_permutation.argtypes = [c.c_uint64, c.c_uint32, c.c_void_p]
            lib.syn_markov_table.argtypes = [c.c_uint64, c.c_double, c.c_void_p]
            lib.syn_genome.argtypes = [c.c_uint64, c.c_uint64, c.c_double, c.c_double, c.c_void_p]
            lib.syn_batch_plan.restype = c.c_uint64
            lib.syn_batch_plan.argtypes = [c.c_uint64, c.c_uint32, c.c_int, c.c_int, c.c_uint64,
                                           c.c_void_p, c.c_uint32, c.c_void_p, c.c_void_p,
                                           c.c_void_p, c.c_void_p]
            lib.syn_words.argtypes = [c.c_uint64, c.c_uint64, c.c_void_p]
            _lib = lib
    return _lib


def _out(n, width, addr):
    if addr is None:
        a = np.empty(n, dtype=_WIDTH_DT[width])
        return a, a.ctypes.data
    return None, addr


def uniform(seed: int, n: int, sigma: int, width: int, addr: int | None = None):
    """i.i.d. uniform symbols in [0, sigma)."""
    a, p = _out(n, width, addr)
    _load().syn_uniform(seed, n, sigma, width, p)
    return a


def zipf(seed: int, n: int, sigma: int, s: float, width: int, addr: int | None = None):
    """Zipf(s) over ranks 1..sigma mapped through a seeded permutation."""
    a, p = _out(n, width, addr)
    if _load().syn_zipf(seed, n, sigma, s, width, p):
        raise MemoryError("zipf table")
    return a


def permutation(seed: int, sigma: int) -> np.ndarray:
    p = np.empty(sigma, dtype=np.uint32)
    _load().syn_permutation(seed, sigma, p.ctypes.data)
    return p


def markov_table(seed: int, alpha: float = 0.5) -> np.ndarray:
    cum = np.empty((64, 4), dtype=np.float64)
    _load().syn_markov_table(seed, alpha, cum.ctypes.data)
    return cum


def genome(seed: int, n: int, alpha: float = 0.5, mean_burst: float = 8.0,
           addr: int | None = None):
    """Order-3 Markov text over {0..3} with geometric bursts; sentinel 4 at n-1."""
    a, p = _out(n, 1, addr)
    _load().syn_genome(seed, n, alpha, 1.0 / mean_burst, p)
    return a


def batch_plan(seed: int, m: int = 4096, lo_log2: int = 10, hi_log2: int = 24,
               cap: int = 1 << 31, sigmas=(4, 256, 4096, 65536)):
    """Lengths, alphabets, zipf flags and seeds of a batched workload."""
    sg = np.ascontiguousarray(sigmas, dtype=np.uint32)
    ln = np.empty(m, dtype=np.uint64)
    sig = np.empty(m, dtype=np.uint32)
    zf = np.empty(m, dtype=np.uint8)
    sd = np.empty(m, dtype=np.uint64)
    total = _load().syn_batch_plan(seed, m, lo_log2, hi_log2, cap, sg.ctypes.data, sg.size,
                                   ln.ctypes.data, sig.ctypes.data, zf.ctypes.data,
                                   sd.ctypes.data)
    return ln, sig, zf.astype(bool), sd, int(total)


def words(seed: int, n: int) -> np.ndarray:
    w = np.empty(n, dtype=np.uint64)
    _load().syn_words(seed, n, w.ctypes.data)
    return w


def queries(seed: int, S: np.ndarray, sigma: int, q: int, invalid_frac: float = 0.01):
    """Mixed access/rank/select arguments: op (0/1/2), c, arg (i or k).

    A third of each op; i uniform in [0, n); c uniform; select draws c
    from the present symbols and k uniform in [1, count_c]; a fraction of
    the queries get out-of-range arguments."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = S.size
    hist = np.bincount(np.asarray(S, dtype=np.int64), minlength=sigma)
    present = np.nonzero(hist)[0]
    op = rng.integers(0, 3, size=q, dtype=np.int64).astype(np.uint8)
    c = rng.integers(0, sigma, size=q, dtype=np.int64).astype(np.uint32)
    arg = rng.integers(0, max(n, 1), size=q, dtype=np.int64).astype(np.uint64)
    sel = op == 2
    if present.size:
        cs = present[rng.integers(0, present.size, size=int(sel.sum()))]
        c[sel] = cs.astype(np.uint32)
        kk = (rng.random(int(sel.sum())) * hist[cs]).astype(np.uint64) + 1
        arg[sel] = np.minimum(kk, hist[cs].astype(np.uint64))
    bad = rng.random(q) < invalid_frac
    kind = rng.integers(0, 3, size=q)
    arg[bad & (op != 2)] = np.uint64(n) + arg[bad & (op != 2)] % np.uint64(7)
    c[bad & (kind == 1)] = np.uint32(sigma)
    arg[bad & (op == 2) & (kind == 0)] = 0
    arg[bad & (op == 2) & (kind == 2)] = np.uint64(n + 1)
    return op, c, arg
