"""GB300-native levelwise wavelet-tree / wavelet-matrix construction.

Thin Python binding over the C ABI in ``include/wavelet.h`` (the shared
library ``libwavelet.so`` built from ``csrc/`` for sm_103a).  The binding only
marshals arguments: every step of a build or a query runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwavelet.so")

WT_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "symbol >= sigma", 3: "out of device memory",
          4: "CUDA error", 5: "not finished yet", 6: "unsupported"}
KIND_WT, KIND_WM, KIND_HUFF, KIND_MULTI, KIND_RS = range(5)
FLAG_NO_DIRECTORY = 1
FLAG_SELECT_O1 = 2

#: every entry point declared in include/wavelet.h
ABI_SYMBOLS = ("wt_build", "wm_build", "wm_build_host", "huff_wt_build", "multiary_build", "rs_build",
               "wt_access", "wt_rank", "wt_select", "wt_sync", "wt_export", "wt_free",
               "wt_symbol_levels", "wt_status_str", "wt_memcpy_d2h", "wt_huffman_lengths",
               "wt_canonical_codes", "wt_prof_enable", "wt_prof_read", "rs_dir_build_static",
               "wm_batch_build", "wm_autotune", "wm_autotune_clear", "wt_query_multi",
               "wt_server_create", "wt_server_submit_build", "wt_server_submit_queries",
               "wt_server_poll", "wt_server_handle", "wt_server_release", "wt_server_stats",
               "wt_server_destroy", "wt_export_select", "wt_dd_merge", "wm_autotune_config",
               "wm_tuning", "wm_batch_build_one", "wt_batch_handle", "wt_batch_sync",
               "wt_batch_free")


class WaveletError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


class BuildOpts(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_uint32), ("tile_symbols", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("k_chunks", ctypes.c_uint32),
                ("select_sample", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class ExportView(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("levels", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("sigma", ctypes.c_uint32), ("bits_per_elem", ctypes.c_uint32),
                ("dir_words_per_rec", ctypes.c_uint32), ("max_code_len", ctypes.c_uint32),
                ("bits", ctypes.c_void_p), ("dir", ctypes.c_void_p), ("samp", ctypes.c_void_p),
                ("level_len", ctypes.POINTER(ctypes.c_uint64)),
                ("level_off", ctypes.POINTER(ctypes.c_uint64)),
                ("dir_off", ctypes.POINTER(ctypes.c_uint64)),
                ("samp_off", ctypes.POINTER(ctypes.c_uint64)),
                ("zeros", ctypes.POINTER(ctypes.c_uint64)),
                ("code_len", ctypes.POINTER(ctypes.c_uint8)),
                ("code", ctypes.POINTER(ctypes.c_uint32))]


class SelectView(ctypes.Structure):
    _fields_ = [("nranges", ctypes.c_uint64), ("nhuge", ctypes.c_uint64),
                ("nsparse", ctypes.c_uint64), ("desc", ctypes.c_void_p), ("sub", ctypes.c_void_p),
                ("sparse", ctypes.c_void_p), ("huge", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_uint32), ("tile_symbols", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("k_chunks", ctypes.c_uint64), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"tau": int(self.tau), "tile_symbols": int(self.tile_symbols),
                "ctas_per_sm": int(self.ctas_per_sm), "k_chunks": int(self.k_chunks),
                "ms": float(self.ms)}


class BatchItem(ctypes.Structure):
    _fields_ = [("d_seq", ctypes.c_void_p), ("n", ctypes.c_uint64), ("sigma", ctypes.c_uint32),
                ("width_bytes", ctypes.c_uint32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_batch_builds", ctypes.c_uint32),
                ("max_batch_queries", ctypes.c_uint32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("kind", ctypes.c_uint32),
                ("submit_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("used_bytes", "budget_bytes", "build_batches", "query_launches",
                 "pending_builds", "pending_queries", "structures")]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libwavelet.so; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (no CPU fallback)")
    lib = ctypes.CDLL(path)
    c = ctypes
    vp, u64, u32 = c.c_void_p, c.c_uint64, c.c_uint32
    hp = c.POINTER(c.c_void_p)
    for name in ("wt_build", "wm_build", "wm_build_host"):
        f = getattr(lib, name)
        f.restype = c.c_int
        f.argtypes = [vp, u64, u32, u32, c.POINTER(BuildOpts), vp, hp]
    lib.huff_wt_build.restype = c.c_int
    lib.huff_wt_build.argtypes = [vp, u64, u32, u32, vp, c.POINTER(BuildOpts), vp, hp]
    lib.multiary_build.restype = c.c_int
    lib.multiary_build.argtypes = [vp, u64, u32, u32, u32, c.POINTER(BuildOpts), vp, hp]
    lib.rs_build.restype = c.c_int
    lib.rs_build.argtypes = [vp, u64, c.POINTER(BuildOpts), vp, hp]
    lib.wt_access.restype = c.c_int
    lib.wt_access.argtypes = [vp, vp, u64, vp, vp]
    lib.wt_rank.restype = c.c_int
    lib.wt_rank.argtypes = [vp, vp, vp, u64, vp, vp]
    lib.wt_select.restype = c.c_int
    lib.wt_select.argtypes = [vp, vp, vp, u64, vp, vp]
    lib.wt_sync.restype = c.c_int
    lib.wt_sync.argtypes = [vp]
    lib.wt_export.restype = c.c_int
    lib.wt_export.argtypes = [vp, c.POINTER(ExportView)]
    lib.wt_free.restype = c.c_int
    lib.wt_free.argtypes = [vp]
    lib.wt_symbol_levels.restype = u64
    lib.wt_symbol_levels.argtypes = [vp]
    lib.wt_status_str.restype = c.c_char_p
    lib.wt_status_str.argtypes = [c.c_int]
    lib.wt_memcpy_d2h.restype = c.c_int
    lib.wt_memcpy_d2h.argtypes = [vp, vp, u64]
    lib.wt_huffman_lengths.restype = u32
    lib.wt_huffman_lengths.argtypes = [vp, u32, u32, vp]
    lib.wt_canonical_codes.restype = None
    lib.wt_canonical_codes.argtypes = [vp, u32, vp]
    lib.rs_dir_build_static.restype = c.c_int
    lib.rs_dir_build_static.argtypes = [vp, u64, vp, vp, vp, vp]
    lib.wt_export_select.restype = c.c_int
    lib.wt_export_select.argtypes = [vp, u32, u32, c.POINTER(SelectView)]
    lib.wt_dd_merge.restype = c.c_int
    lib.wt_dd_merge.argtypes = [hp, u32, c.POINTER(BuildOpts), vp, hp]
    lib.wm_batch_build.restype = c.c_int
    lib.wm_batch_build.argtypes = [c.POINTER(BatchItem), u32, c.POINTER(BuildOpts), vp, hp]
    lib.wm_autotune.restype = c.c_int
    lib.wm_autotune.argtypes = [vp, u64, u32, u32, vp, c.POINTER(u32), c.POINTER(c.c_float)]
    lib.wm_batch_build_one.restype = c.c_int
    lib.wm_batch_build_one.argtypes = [c.POINTER(BatchItem), u32, c.POINTER(BuildOpts), vp, hp]
    lib.wt_batch_handle.restype = vp
    lib.wt_batch_handle.argtypes = [vp, u32]
    lib.wt_batch_sync.restype = c.c_int
    lib.wt_batch_sync.argtypes = [vp, vp]
    lib.wt_batch_free.restype = c.c_int
    lib.wt_batch_free.argtypes = [vp]
    lib.wm_autotune_config.restype = c.c_int
    lib.wm_autotune_config.argtypes = [vp, u64, u32, u32, vp, c.POINTER(Tuning)]
    lib.wm_tuning.restype = c.c_int
    lib.wm_tuning.argtypes = [u64, u32, c.POINTER(Tuning)]
    lib.wm_autotune_clear.restype = None
    lib.wm_autotune_clear.argtypes = []
    lib.wt_query_multi.restype = c.c_int
    lib.wt_query_multi.argtypes = [hp, u32, vp, vp, vp, vp, u64, vp, vp]
    lib.wt_server_create.restype = c.c_int
    lib.wt_server_create.argtypes = [c.POINTER(ServerOpts), hp]
    lib.wt_server_submit_build.restype = c.c_int
    lib.wt_server_submit_build.argtypes = [vp, vp, u64, u32, u32, c.POINTER(u64)]
    lib.wt_server_submit_queries.restype = c.c_int
    lib.wt_server_submit_queries.argtypes = [vp, u64, vp, vp, vp, vp, c.POINTER(u64)]
    lib.wt_server_poll.restype = c.c_int
    lib.wt_server_poll.argtypes = [vp, u64, c.c_int, vp, c.POINTER(RequestInfo)]
    lib.wt_server_handle.restype = c.c_int
    lib.wt_server_handle.argtypes = [vp, u64, hp]
    lib.wt_server_release.restype = c.c_int
    lib.wt_server_release.argtypes = [vp, u64]
    lib.wt_server_stats.restype = c.c_int
    lib.wt_server_stats.argtypes = [vp, c.POINTER(ServerStats)]
    lib.wt_server_destroy.restype = c.c_int
    lib.wt_server_destroy.argtypes = [vp]
    lib.wt_prof_enable.restype = None
    lib.wt_prof_enable.argtypes = [c.c_int]
    lib.wt_prof_read.restype = c.c_int
    lib.wt_prof_read.argtypes = [c.POINTER(u64), c.POINTER(u64), c.POINTER(c.c_double)]
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != WT_OK:
        raise WaveletError(status, what)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _opts(tau=0, ctas_per_sm=0, flags=0, tile_symbols=0):
    o = BuildOpts()
    o.tau, o.ctas_per_sm, o.flags, o.tile_symbols = tau, ctas_per_sm, flags, tile_symbols
    return o


def _ptr(x) -> int:
    return x if isinstance(x, int) else x.data_ptr()


def d2h(dptr: int, nbytes: int, dtype=np.uint64) -> np.ndarray:
    """Copy device memory (an exported array) to a new numpy array."""
    itemsize = np.dtype(dtype).itemsize
    out = np.empty(max(nbytes // itemsize, 0), dtype=dtype)
    if nbytes:
        _check(load_library().wt_memcpy_d2h(out.ctypes.data, dptr, nbytes), "wt_memcpy_d2h")
    return out


@dataclass
class Exported:
    kind: int
    levels: int
    n: int
    sigma: int
    bits_per_elem: int
    max_code_len: int
    level_len: np.ndarray
    level_off: np.ndarray
    dir_off: np.ndarray
    samp_off: np.ndarray
    zeros: np.ndarray
    bits: np.ndarray
    dir: np.ndarray
    samp: np.ndarray
    code_len: np.ndarray | None
    code: np.ndarray | None

    def level(self, l: int) -> np.ndarray:
        return self.bits[int(self.level_off[l]):int(self.level_off[l + 1])]

    def level_dir(self, l: int) -> np.ndarray:
        w = 8 if self.bits_per_elem == 2 else 2
        return self.dir[int(self.dir_off[l]):int(self.dir_off[l + 1])].reshape(-1, w)

    def samples(self, l: int, b: int) -> np.ndarray:
        """Positions of occurrences 0, 4096, ... of value b on level l (bit
        value; digit value on the digit levels of a 4-ary tree)."""
        if self.bits_per_elem == 2:
            cnt = int(self.level_dir(l)[-1, b])
            s = int(self.samp_off[4 * l + b])
        else:
            n = int(self.level_len[l])
            z = int(self.zeros[l])
            cnt = z if b == 0 else n - z
            s = int(self.samp_off[2 * l + b])
        return self.samp[s:s + (cnt + 4095) // 4096]


class Handle:
    """A built structure; owns its device arrays until ``free()``."""

    def __init__(self, raw: ctypes.c_void_p, keep=None):
        self._h = raw
        self._keep = keep  # caller buffer that must outlive the handle (rs_build)

    @property
    def raw(self):
        return self._h

    def _live(self):
        if not self._h:
            raise WaveletError(1, "handle already freed")
        return self._h

    def sync(self):
        _check(load_library().wt_sync(self._live()), "wt_sync")

    def symbol_levels(self) -> int:
        return int(load_library().wt_symbol_levels(self._live()))

    def access(self, i, out, q=None, stream=None):
        q = i.numel() if q is None else q
        _check(load_library().wt_access(self._live(), _ptr(i), q, _ptr(out), _stream_ptr(stream)),
               "wt_access")
        return out

    def rank(self, c, i, out, q=None, stream=None):
        q = i.numel() if q is None else q
        _check(load_library().wt_rank(self._live(), _ptr(c), _ptr(i), q, _ptr(out),
                                      _stream_ptr(stream)), "wt_rank")
        return out

    def select(self, c, k, out, q=None, stream=None):
        q = k.numel() if q is None else q
        _check(load_library().wt_select(self._live(), _ptr(c), _ptr(k), q, _ptr(out),
                                        _stream_ptr(stream)), "wt_select")
        return out

    def export(self) -> Exported:
        v = ExportView()
        _check(load_library().wt_export(self._live(), ctypes.byref(v)), "wt_export")
        L = v.levels

        def host(p, n, dt=np.uint64):
            if n == 0 or not p:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(p, shape=(n,)).astype(dt).copy()

        level_len = host(v.level_len, L)
        level_off = host(v.level_off, L + 1)
        dir_off = host(v.dir_off, L + 1)
        samp_off = host(v.samp_off, (4 if v.bits_per_elem == 2 else 2) * L + 1)
        zeros = host(v.zeros, L)
        nw = int(level_off[-1]) if L else 0
        bits = d2h(v.bits, nw * 8) if nw else np.zeros(0, np.uint64)
        nd = int(dir_off[-1]) if L else 0
        dirs = d2h(v.dir, nd * 8) if nd else np.zeros(0, np.uint64)
        ns = int(samp_off[-1]) if L else 0
        samp = d2h(v.samp, ns * 8) if ns else np.zeros(0, np.uint64)
        code_len = host(v.code_len, v.sigma, np.uint8) if v.code_len else None
        code = host(v.code, v.sigma, np.uint32) if v.code else None
        return Exported(v.kind, L, v.n, v.sigma, v.bits_per_elem, v.max_code_len, level_len,
                        level_off, dir_off, samp_off, zeros, bits, dirs, samp, code_len, code)

    def export_select(self, level: int, bit: int):
        """Arrays of the constant-time select directory of one level and bit
        value (desc, sub, sparse, huge), copied to the host."""
        v = SelectView()
        _check(load_library().wt_export_select(self._live(), level, bit, ctypes.byref(v)),
               "wt_export_select")
        R, H, S = int(v.nranges), int(v.nhuge), int(v.nsparse)
        desc = d2h(v.desc, 8 * R)
        sub = d2h(v.sub, 4 * 16 * R, np.uint32)
        sparse = d2h(v.sparse, 4 * 256 * S, np.uint32)
        huge = d2h(v.huge, 8 * 4096 * H)
        return desc, sub, sparse, huge

    def free(self):
        if self._h:
            _check(load_library().wt_free(self._h), "wt_free")
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.wt_free(self._h)
        except Exception:
            pass


def _width(seq) -> int:
    return seq.element_size()


def _build(fn, what, *args):
    h = ctypes.c_void_p()
    _check(fn(*args, ctypes.byref(h)), what)
    return Handle(h)


def wm_build(seq, sigma: int, n: int | None = None, tau: int = 0, ctas_per_sm: int = 0,
             flags: int = 0, stream=None, tile_symbols: int = 0) -> Handle:
    """Wavelet matrix of a device tensor of uint8/int16/int32 symbols."""
    n = seq.numel() if n is None else n
    o = _opts(tau, ctas_per_sm, flags, tile_symbols)
    return _build(load_library().wm_build, "wm_build", _ptr(seq), n, sigma, _width(seq),
                  ctypes.byref(o), _stream_ptr(stream))


def wm_build_host(seq, sigma: int, n: int | None = None, tau: int = 0, ctas_per_sm: int = 0,
                  flags: int = 0, stream=None, tile_symbols: int = 0) -> Handle:
    """Wavelet matrix of a host tensor (ideally pinned) or numpy array of
    uint8/int16/int32 symbols: the library copies it to the device on the
    stream and builds there."""
    if isinstance(seq, np.ndarray):
        ptr, width, count = seq.ctypes.data, seq.itemsize, seq.size
    else:
        if seq.is_cuda:
            raise ValueError("wm_build_host takes host memory; use wm_build for device tensors")
        ptr, width, count = seq.data_ptr(), seq.element_size(), seq.numel()
    n = count if n is None else n
    if n > count:
        raise ValueError(f"n = {n} exceeds the {count} host elements")
    o = _opts(tau, ctas_per_sm, flags, tile_symbols)
    return _build(load_library().wm_build_host, "wm_build_host", ptr, n, sigma, width,
                  ctypes.byref(o), _stream_ptr(stream))


def wt_build(seq, sigma: int, n: int | None = None, tau: int = 0, ctas_per_sm: int = 0,
             flags: int = 0, stream=None) -> Handle:
    """Balanced levelwise wavelet tree."""
    n = seq.numel() if n is None else n
    o = _opts(tau, ctas_per_sm, flags)
    return _build(load_library().wt_build, "wt_build", _ptr(seq), n, sigma, _width(seq),
                  ctypes.byref(o), _stream_ptr(stream))


def huff_wt_build(seq, sigma: int, code_len: np.ndarray | None = None, n: int | None = None,
                  tau: int = 0, flags: int = 0, stream=None) -> Handle:
    """Huffman-shaped wavelet tree (lengths from the histogram when code_len is None)."""
    n = seq.numel() if n is None else n
    o = _opts(tau, 0, flags)
    cl = None
    if code_len is not None:
        cl = np.ascontiguousarray(code_len, dtype=np.uint8)
    h = ctypes.c_void_p()
    _check(load_library().huff_wt_build(_ptr(seq), n, sigma, _width(seq),
                                         cl.ctypes.data if cl is not None else None,
                                         ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)),
           "huff_wt_build")
    return Handle(h)


def multiary_build(seq, sigma: int, degree: int = 4, n: int | None = None, tau: int = 0,
                   flags: int = 0, stream=None) -> Handle:
    """4-ary wavelet tree (2-bit digit levels)."""
    n = seq.numel() if n is None else n
    o = _opts(tau, 0, flags)
    h = ctypes.c_void_p()
    _check(load_library().multiary_build(_ptr(seq), n, sigma, _width(seq), degree,
                                          ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)),
           "multiary_build")
    return Handle(h)


def rs_build(bits, nbits: int, flags: int = 0, stream=None) -> Handle:
    """Rank/select directory over a device bitvector (kept referenced by the handle)."""
    o = _opts(flags=flags)
    h = ctypes.c_void_p()
    _check(load_library().rs_build(_ptr(bits), nbits, ctypes.byref(o), _stream_ptr(stream),
                                    ctypes.byref(h)), "rs_build")
    return Handle(h, keep=bits)


def rs_dir_build_static(bits, nbits: int, dir_out, samp0_out, samp1_out, stream=None):
    """Rank directory and select samples of a device bitvector into caller
    buffers, with no device allocation (scratch in a static device array;
    nbits <= 2^30; calls must not overlap on the GPU)."""
    _check(load_library().rs_dir_build_static(_ptr(bits), nbits, _ptr(dir_out), _ptr(samp0_out),
                                               _ptr(samp1_out), _stream_ptr(stream)),
           "rs_dir_build_static")


def prof_enable(on: bool = True):
    """Count kernel launches and time partition-pass launches (CUDA events)."""
    load_library().wt_prof_enable(1 if on else 0)


def prof_read():
    """(kernel launches, pass launches, summed pass milliseconds) since prof_enable."""
    a, b, ms = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(load_library().wt_prof_read(ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)),
           "wt_prof_read")
    return int(a.value), int(b.value), float(ms.value)


def huffman_lengths(hist: np.ndarray, cap: int = 32):
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    ln = np.zeros(h.size, dtype=np.uint8)
    mx = load_library().wt_huffman_lengths(h.ctypes.data, h.size, cap, ln.ctypes.data)
    return ln, int(mx)


def canonical_codes(lengths: np.ndarray) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(ln.size, dtype=np.uint32)
    load_library().wt_canonical_codes(ln.ctypes.data, ln.size, code.ctypes.data)
    return code


def wm_batch_build(seqs, sigmas, ns=None, tau: int = 0, flags: int = 0, stream=None):
    """Wavelet matrices of several device tensors with one batched build.

    Returns one Handle per sequence (they share one device allocation)."""
    m = len(seqs)
    items = (BatchItem * max(m, 1))()
    for i, (sq, sg) in enumerate(zip(seqs, sigmas)):
        items[i].d_seq = _ptr(sq) if sq is not None else 0
        items[i].n = sq.numel() if ns is None else int(ns[i])
        items[i].sigma = int(sg)
        items[i].width_bytes = _width(sq) if sq is not None else 2
    outs = (ctypes.c_void_p * max(m, 1))()
    o = _opts(tau, 0, flags)
    _check(load_library().wm_batch_build(items, m, ctypes.byref(o), _stream_ptr(stream), outs),
           "wm_batch_build")
    return [Handle(ctypes.c_void_p(outs[i])) for i in range(m)]


class _BatchMember(Handle):
    """A structure of a Batch: usable like a Handle, released with its batch."""

    def free(self):
        self._h = None

    def __del__(self):
        pass


class Batch:
    """The structures of one batched build behind one object (wm_batch_build_one)."""

    def __init__(self, raw: ctypes.c_void_p, m: int):
        self._b = raw
        self._m = m

    def __len__(self):
        return self._m

    def handle(self, i: int) -> Handle:
        if not self._b:
            raise WaveletError(1, "batch already freed")
        h = load_library().wt_batch_handle(self._b, i)
        if not h:
            raise WaveletError(1, "wt_batch_handle")
        return _BatchMember(ctypes.c_void_p(h))

    def sync(self) -> np.ndarray:
        """Wait once; the status of every sequence (0 = built)."""
        st = np.zeros(max(self._m, 1), dtype=np.int32)
        load_library().wt_batch_sync(self._b, st.ctypes.data)
        return st[:self._m]

    def free(self):
        if self._b:
            _check(load_library().wt_batch_free(self._b), "wt_batch_free")
            self._b = None

    def __del__(self):
        try:
            if self._b and _lib is not None:
                _lib.wt_batch_free(self._b)
        except Exception:
            pass


_ITEM_DT = np.dtype([("d_seq", np.uint64), ("n", np.uint64), ("sigma", np.uint32),
                     ("width_bytes", np.uint32)])


def batch_items(base_ptr: int, byte_offsets, ns, sigmas, width: int = 2):
    """wt_batch_item array for sequences at base_ptr + byte_offsets[i] (device
    addresses), filled with numpy (no per-sequence Python work)."""
    m = len(ns)
    a = np.zeros(max(m, 1), dtype=_ITEM_DT)
    a["d_seq"][:m] = np.uint64(base_ptr) + np.asarray(byte_offsets, dtype=np.uint64)[:m]
    a["n"][:m] = np.asarray(ns, dtype=np.uint64)
    a["sigma"][:m] = np.asarray(sigmas, dtype=np.uint32)
    a["width_bytes"][:m] = width
    return a


def wm_batch_build_one(seqs=None, sigmas=None, ns=None, tau: int = 0, flags: int = 0,
                       stream=None, items=None) -> Batch:
    """wm_batch_build as one Batch object (one object per step instead of m).
    Either device tensors and sigmas, or a prebuilt batch_items() array."""
    if items is None:
        m = len(seqs)
        items = np.zeros(max(m, 1), dtype=_ITEM_DT)
        for i, (sq, sg) in enumerate(zip(seqs, sigmas)):
            items[i] = (_ptr(sq) if sq is not None else 0,
                        sq.numel() if ns is None else int(ns[i]), int(sg),
                        _width(sq) if sq is not None else 2)
    else:
        m = int(np.count_nonzero(items["sigma"])) if ns is None else int(ns)
    b = ctypes.c_void_p()
    o = _opts(tau, 0, flags)
    ip = ctypes.cast(items.ctypes.data, ctypes.POINTER(BatchItem))
    _check(load_library().wm_batch_build_one(ip, m, ctypes.byref(o), _stream_ptr(stream),
                                              ctypes.byref(b)), "wm_batch_build_one")
    return Batch(b, m)


def dd_merge(parts, flags: int = 0, stream=None) -> Handle:
    """The structure of the concatenation of consecutive pieces of one
    sequence from the pieces' structures (all wavelet matrices or all
    balanced wavelet trees, same sigma): domain-decomposition merge."""
    r = len(parts)
    arr = (ctypes.c_void_p * max(r, 1))()
    for i, p in enumerate(parts):
        arr[i] = p._live()
    h = ctypes.c_void_p()
    o = _opts(0, 0, flags)
    _check(load_library().wt_dd_merge(arr, r, ctypes.byref(o), _stream_ptr(stream),
                                       ctypes.byref(h)), "wt_dd_merge")
    return Handle(h)


def wm_autotune(seq, sigma: int, n: int | None = None, stream=None):
    """Time tau = 1..min(8, L) on this sequence; returns (best tau, ms per tau)
    and records the choice for later builds with tau = 0."""
    n = seq.numel() if n is None else n
    best = ctypes.c_uint32()
    ms = (ctypes.c_float * 8)()
    _check(load_library().wm_autotune(_ptr(seq), n, sigma, _width(seq), _stream_ptr(stream),
                                       ctypes.byref(best), ms), "wm_autotune")
    return int(best.value), [float(v) for v in ms]


def wm_autotune_config(seq, sigma: int, n: int | None = None, stream=None) -> dict:
    """Tune (tau, tile size, CTAs per SM) on this sequence; returns the
    fastest configuration (with K and its build time) and records it for
    later builds with zero options."""
    n = seq.numel() if n is None else n
    t = Tuning()
    _check(load_library().wm_autotune_config(_ptr(seq), n, sigma, _width(seq),
                                              _stream_ptr(stream), ctypes.byref(t)),
           "wm_autotune_config")
    return t.as_dict()


def wm_tuning(n: int, sigma: int) -> dict:
    """The configuration a wm_build with zero options takes."""
    t = Tuning()
    _check(load_library().wm_tuning(n, sigma, ctypes.byref(t)), "wm_tuning")
    return t.as_dict()


def wm_autotune_clear():
    load_library().wm_autotune_clear()


def query_multi(handles, sid, op, c, x, out, q=None, stream=None):
    """One launch of queries over several structures (device tensors:
    sid u32, op u8, c u32, x u64, out u64)."""
    q = x.numel() if q is None else q
    hs = (ctypes.c_void_p * max(len(handles), 1))()
    for i, h in enumerate(handles):
        hs[i] = h._live().value
    _check(load_library().wt_query_multi(hs, len(handles), _ptr(sid), _ptr(op), _ptr(c), _ptr(x),
                                          q, _ptr(out), _stream_ptr(stream)), "wt_query_multi")
    return out


class Server:
    """Serving loop of the library (wt_server_*): builds of host sequences and
    query batches over built structures, continuously batched on the GPU."""

    def __init__(self, budget_bytes: int, max_batch_builds: int = 0, max_batch_queries: int = 0):
        o = ServerOpts()
        o.budget_bytes, o.max_batch_builds, o.max_batch_queries = (budget_bytes, max_batch_builds,
                                                                   max_batch_queries)
        self._s = ctypes.c_void_p()
        _check(load_library().wt_server_create(ctypes.byref(o), ctypes.byref(self._s)),
               "wt_server_create")

    def submit_build(self, seq: np.ndarray, sigma: int) -> int:
        a = np.ascontiguousarray(seq)
        r = ctypes.c_uint64()
        _check(load_library().wt_server_submit_build(self._s, a.ctypes.data, a.size, sigma,
                                                      a.dtype.itemsize, ctypes.byref(r)),
               "wt_server_submit_build")
        return int(r.value)

    def submit_queries(self, sid, op, c, x) -> int:
        sid = np.ascontiguousarray(sid, dtype=np.uint64)
        op = np.ascontiguousarray(op, dtype=np.uint8)
        c = np.ascontiguousarray(c, dtype=np.uint32)
        x = np.ascontiguousarray(x, dtype=np.uint64)
        r = ctypes.c_uint64()
        _check(load_library().wt_server_submit_queries(self._s, sid.size, sid.ctypes.data,
                                                        op.ctypes.data, c.ctypes.data,
                                                        x.ctypes.data, ctypes.byref(r)),
               "wt_server_submit_queries")
        return int(r.value)

    def poll(self, req: int, q: int = 0, wait: bool = True):
        """(status, submit_ns, done_ns, answers or None); status None while running."""
        out = np.zeros(q, dtype=np.uint64) if q else None
        info = RequestInfo()
        st = load_library().wt_server_poll(self._s, req, 1 if wait else 0,
                                           out.ctypes.data if q else None, ctypes.byref(info))
        if st == 5 and not wait:
            return None, info.submit_ns, 0, None
        _check(st, "wt_server_poll")
        return info.status, info.submit_ns, info.done_ns, out

    def handle(self, sid: int):
        h = ctypes.c_void_p()
        _check(load_library().wt_server_handle(self._s, sid, ctypes.byref(h)), "wt_server_handle")
        return h

    def release(self, sid: int):
        _check(load_library().wt_server_release(self._s, sid), "wt_server_release")

    def stats(self) -> dict:
        st = ServerStats()
        _check(load_library().wt_server_stats(self._s, ctypes.byref(st)), "wt_server_stats")
        return {k: int(getattr(st, k)) for k, _ in ServerStats._fields_}

    def close(self):
        if self._s:
            load_library().wt_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
