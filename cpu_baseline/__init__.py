"""Multi-threaded CPU constructions of the wavelet matrix with its rank
directories and select samples (wm_cpu.cpp): levelwise splits, and big
levels with table-driven packed short lists (Section 3, Theorem 4.1); the
benchmark's timed CPU comparisons.  Not used by the library."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wm_cpu.cpp")
_SO = os.path.join(_HERE, "libwm_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", _SO])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.cpu_wm_build.restype = ctypes.c_int
        lib.cpu_wm_build.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
        lib.cpu_wm_build_short.restype = ctypes.c_int
        lib.cpu_wm_build_short.argtypes = lib.cpu_wm_build.argtypes
        _lib = lib
    return _lib


def wm_build(S: np.ndarray, L: int, threads: int, short_lists: bool = False):
    """Level words (L, W), zero counts (L,), rank records (L, nsb+1, 2) and
    select samples (L, 2, n/4096 + 1) of the wavelet matrix of uint16 S.
    short_lists: big levels every 4 levels and table-driven short lists in
    between (Section 3, Theorem 4.1) instead of one split per level."""
    S = np.ascontiguousarray(S, dtype=np.uint16)
    n = S.size
    W = ((n + 2047) // 2048) * 32
    nsb = (n + 2047) // 2048
    cap = n // 4096 + 1
    bits = np.zeros((L, W), dtype=np.uint64)
    zeros = np.zeros(L, dtype=np.uint64)
    dirs = np.zeros((L, nsb + 1, 2), dtype=np.uint64)
    samp = np.zeros((L, 2, cap), dtype=np.uint64)
    fn = _load().cpu_wm_build_short if short_lists else _load().cpu_wm_build
    fn(S.ctypes.data, n, L, threads, bits.ctypes.data, zeros.ctypes.data, dirs.ctypes.data,
       samp.ctypes.data)
    return bits, zeros, dirs, samp
