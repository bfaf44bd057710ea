"""CPU oracle for levelwise wavelet-tree / wavelet-matrix construction.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1610_03524_gb300``) never imports it, and this package imports
nothing from the product path.

The arithmetic lives in ``wt_oracle.c`` (plain C, single-threaded, one
function per definition of Shun's paper); this module only compiles it with
``gcc`` and marshals numpy arrays through ``ctypes``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wt_oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U64P = ctypes.POINTER(ctypes.c_uint64)
U32P = ctypes.POINTER(ctypes.c_uint32)
U8P = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no -march flags: same results on x86 and Arm)."""
    stale = (not os.path.exists(_SO)) or any(
        os.path.getmtime(p) > os.path.getmtime(_SO) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.orc_levels.restype = ctypes.c_uint32
            lib.orc_levels.argtypes = [ctypes.c_uint32]
            lib.orc_level_words.restype = ctypes.c_uint64
            lib.orc_level_words.argtypes = [ctypes.c_uint64]
            lib.orc_wt_build.argtypes = [U32P, ctypes.c_uint64, ctypes.c_uint32, U64P]
            lib.orc_wm_build.argtypes = [U32P, ctypes.c_uint64, ctypes.c_uint32, U64P, U64P]
            lib.orc_rank_dir.argtypes = [U64P, ctypes.c_uint64, U64P]
            lib.orc_select_samples.restype = ctypes.c_uint64
            lib.orc_select_samples.argtypes = [U64P, ctypes.c_uint64, ctypes.c_uint32, U64P]
            lib.orc_clark_build.restype = ctypes.c_int
            lib.orc_clark_build.argtypes = [U64P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_uint64, U64P, U64P, U64P, U64P, U32P, U32P,
                                            U64P]
            lib.orc_clark_digits.restype = ctypes.c_int
            lib.orc_clark_digits.argtypes = lib.orc_clark_build.argtypes
            lib.orc_digit_samples.restype = ctypes.c_uint64
            lib.orc_digit_samples.argtypes = [U64P, ctypes.c_uint64, ctypes.c_uint32, U64P]
            lib.orc_huffman_lengths.restype = ctypes.c_uint32
            lib.orc_huffman_lengths.argtypes = [U64P, ctypes.c_uint32, ctypes.c_uint32, U8P]
            lib.orc_canonical_codes.argtypes = [U8P, ctypes.c_uint32, U32P]
            lib.orc_huff_level_sizes.argtypes = [U32P, ctypes.c_uint64, U8P, ctypes.c_uint32, U64P]
            lib.orc_huff_wt_build.argtypes = [U32P, ctypes.c_uint64, U8P, U32P, ctypes.c_uint32,
                                              U64P, U64P]
            lib.orc_mwt_build.argtypes = [U32P, ctypes.c_uint64, ctypes.c_uint32, U64P]
            lib.orc_mwt_dir.argtypes = [U64P, ctypes.c_uint64, U64P]
            lib.orc_access.argtypes = [U32P, ctypes.c_uint64, U64P, ctypes.c_uint64, U64P]
            lib.orc_rank.argtypes = [U32P, ctypes.c_uint64, ctypes.c_uint32, U32P, U64P,
                                     ctypes.c_uint64, U64P]
            lib.orc_select.argtypes = [U32P, ctypes.c_uint64, ctypes.c_uint32, U32P, U64P,
                                       ctypes.c_uint64, U64P]
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(t)


def _u32(S) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(S), dtype=np.uint32)


def levels(sigma: int) -> int:
    return int(_load().orc_levels(sigma))


def level_words(nbits: int) -> int:
    return int(_load().orc_level_words(nbits))


def wt_build(S, sigma: int) -> np.ndarray:
    """Balanced WT level bitmaps, shape (L, level_words(n))."""
    S = _u32(S)
    L, W = levels(sigma), level_words(S.size)
    bits = np.zeros((L, W), dtype=np.uint64)
    if _load().orc_wt_build(_p(S, U32P), S.size, sigma, _p(bits, U64P)):
        raise MemoryError("oracle wt_build")
    return bits


def wm_build(S, sigma: int):
    """Wavelet-matrix level bitmaps (L, W) and zero counts (L,)."""
    S = _u32(S)
    L, W = levels(sigma), level_words(S.size)
    bits = np.zeros((L, W), dtype=np.uint64)
    zeros = np.zeros(L, dtype=np.uint64)
    if _load().orc_wm_build(_p(S, U32P), S.size, sigma, _p(bits, U64P), _p(zeros, U64P)):
        raise MemoryError("oracle wm_build")
    return bits, zeros


def rank_dir(bits_level: np.ndarray, nbits: int) -> np.ndarray:
    """Rank records (nsb+1, 2): [zeros_before, packed u16 rel[4]]."""
    b = np.ascontiguousarray(bits_level, dtype=np.uint64)
    nsb = (nbits + 2047) // 2048
    rec = np.zeros((nsb + 1, 2), dtype=np.uint64)
    _load().orc_rank_dir(_p(b, U64P), nbits, _p(rec, U64P))
    return rec


def select_samples(bits_level: np.ndarray, nbits: int, b: int) -> np.ndarray:
    bl = np.ascontiguousarray(bits_level, dtype=np.uint64)
    out = np.zeros(nbits // 4096 + 2, dtype=np.uint64)
    ns = _load().orc_select_samples(_p(bl, U64P), nbits, b, _p(out, U64P))
    return out[:ns].copy()


CLARK_HUGE_MIN = 1 << 32
CLARK_SPARSE_MIN = 1 << 16


def _clark(fn, words, n, v, huge_min, sparse_min):
    bl = np.ascontiguousarray(words, dtype=np.uint64)
    null64 = ctypes.cast(None, U64P)
    null32 = ctypes.cast(None, U32P)
    c = [ctypes.c_uint64() for _ in range(3)]
    if fn(_p(bl, U64P), n, v, huge_min, sparse_min, ctypes.byref(c[0]),
          ctypes.byref(c[1]), ctypes.byref(c[2]), null64, null32, null32, null64):
        raise MemoryError("oracle clark")
    R, H, S = (int(x.value) for x in c)
    desc = np.zeros(max(R, 1), dtype=np.uint64)
    sub = np.zeros(max(16 * R, 1), dtype=np.uint32)
    sparse = np.zeros(max(256 * S, 1), dtype=np.uint32)
    huge = np.zeros(max(4096 * H, 1), dtype=np.uint64)
    if fn(_p(bl, U64P), n, v, huge_min, sparse_min, ctypes.byref(c[0]),
          ctypes.byref(c[1]), ctypes.byref(c[2]), _p(desc, U64P), _p(sub, U32P),
          _p(sparse, U32P), _p(huge, U64P)):
        raise MemoryError("oracle clark")
    return desc[:R], sub[:16 * R], sparse[:256 * S], huge[:4096 * H]


def clark(bits_level: np.ndarray, nbits: int, b: int, huge_min: int = CLARK_HUGE_MIN,
          sparse_min: int = CLARK_SPARSE_MIN):
    """Constant-time select directory of one bit value (desc, sub, sparse, huge)."""
    return _clark(_load().orc_clark_build, bits_level, nbits, b, huge_min, sparse_min)


def clark_digits(dig_level: np.ndarray, ndig: int, d: int, huge_min: int = CLARK_HUGE_MIN,
                 sparse_min: int = CLARK_SPARSE_MIN):
    """The same for the occurrences of digit value d in a 4-ary digit level."""
    return _clark(_load().orc_clark_digits, dig_level, ndig, d, huge_min, sparse_min)


def digit_samples(dig_level: np.ndarray, ndig: int, d: int) -> np.ndarray:
    """Position of every 4096th occurrence of digit value d (from occurrence 0)."""
    dl = np.ascontiguousarray(dig_level, dtype=np.uint64)
    out = np.zeros(ndig // 4096 + 2, dtype=np.uint64)
    ns = _load().orc_digit_samples(_p(dl, U64P), ndig, d, _p(out, U64P))
    return out[:ns].copy()


def huffman_lengths(hist, cap: int = 32):
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    ln = np.zeros(h.size, dtype=np.uint8)
    mx = _load().orc_huffman_lengths(_p(h, U64P), h.size, cap, _p(ln, U8P))
    return ln, int(mx)


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(ln.size, dtype=np.uint32)
    _load().orc_canonical_codes(_p(ln, U8P), ln.size, _p(code, U32P))
    return code


def huff_wt_build(S, lengths, codes):
    """Huffman-shaped WT: (bits concatenated, word offsets (maxlen+1,), level sizes)."""
    S = _u32(S)
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    cd = np.ascontiguousarray(codes, dtype=np.uint32)
    maxlen = int(ln.max()) if ln.size else 0
    nl = np.zeros(max(maxlen, 1), dtype=np.uint64)
    lib = _load()
    lib.orc_huff_level_sizes(_p(S, U32P), S.size, _p(ln, U8P), maxlen, _p(nl, U64P))
    nl = nl[:maxlen]
    woff = np.zeros(maxlen + 1, dtype=np.uint64)
    for l in range(maxlen):
        woff[l + 1] = woff[l] + level_words(int(nl[l]))
    bits = np.zeros(max(int(woff[-1]), 1), dtype=np.uint64)
    if lib.orc_huff_wt_build(_p(S, U32P), S.size, _p(ln, U8P), _p(cd, U32P), maxlen,
                             _p(woff, U64P), _p(bits, U64P)):
        raise MemoryError("oracle huff_wt_build")
    return bits[:int(woff[-1])], woff, nl


def mwt_build(S, sigma: int) -> np.ndarray:
    """4-ary WT digit levels, shape (ceil(L/2), level_words(2n))."""
    S = _u32(S)
    L = levels(sigma)
    D, W = (L + 1) // 2, level_words(2 * S.size)
    dig = np.zeros((D, W), dtype=np.uint64)
    if _load().orc_mwt_build(_p(S, U32P), S.size, sigma, _p(dig, U64P)):
        raise MemoryError("oracle mwt_build")
    return dig


def mwt_dir(dig_level: np.ndarray, ndig: int) -> np.ndarray:
    d = np.ascontiguousarray(dig_level, dtype=np.uint64)
    nsb = (ndig + 1023) // 1024
    rec = np.zeros((nsb + 1, 8), dtype=np.uint64)
    _load().orc_mwt_dir(_p(d, U64P), ndig, _p(rec, U64P))
    return rec


def access(S, i) -> np.ndarray:
    S = _u32(S)
    i = np.ascontiguousarray(i, dtype=np.uint64)
    out = np.zeros(i.size, dtype=np.uint64)
    _load().orc_access(_p(S, U32P), S.size, _p(i, U64P), i.size, _p(out, U64P))
    return out


def rank(S, sigma: int, c, i) -> np.ndarray:
    S = _u32(S)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    i = np.ascontiguousarray(i, dtype=np.uint64)
    out = np.zeros(i.size, dtype=np.uint64)
    _load().orc_rank(_p(S, U32P), S.size, sigma, _p(c, U32P), _p(i, U64P), i.size,
                     _p(out, U64P))
    return out


def select(S, sigma: int, c, k) -> np.ndarray:
    S = _u32(S)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    k = np.ascontiguousarray(k, dtype=np.uint64)
    out = np.zeros(k.size, dtype=np.uint64)
    _load().orc_select(_p(S, U32P), S.size, sigma, _p(c, U32P), _p(k, U64P), k.size,
                       _p(out, U64P))
    return out


def bits_to_str(level: np.ndarray, nbits: int) -> str:
    """Render the first nbits of a level bitmap as a 0/1 string (bit 0 first)."""
    return "".join(str((int(level[i >> 6]) >> (i & 63)) & 1) for i in range(nbits))
