"""C ABI: the library loads without a GPU, exports every declared entry point,
and its host-side logic (Huffman code construction) matches the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03524_gb300 as wt
    return wt


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib.ABI_SYMBOLS)


def test_status_strings(lib):
    so = lib.load_library()
    for s in range(7):
        assert so.wt_status_str(s)


@pytest.mark.parametrize("seed,sigma,s", [(1, 2, 1.0), (2, 17, 1.0), (3, 1000, 1.1), (4, 5000, 0.7),
                                          (5, 1 << 16, 1.0)])
def test_library_huffman_matches_oracle(lib, seed, sigma, s):
    S = synth.zipf(seed, 1 << 16, sigma, s, 4)
    hist = np.bincount(S.astype(np.int64), minlength=sigma).astype(np.uint64)
    la, ma = lib.huffman_lengths(hist, 32)
    lo, mo = oracle.huffman_lengths(hist, 32)
    assert ma == mo and np.array_equal(la, lo)
    assert np.array_equal(lib.canonical_codes(la), oracle.canonical_codes(lo))


def test_library_package_merge_matches_oracle(lib):
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    hist = np.array(fib + [0, 3, 3], dtype=np.uint64)
    for cap in (32, 24, 10, 7):
        la, ma = lib.huffman_lengths(hist, cap)
        lo, mo = oracle.huffman_lengths(hist, cap)
        assert ma == mo <= cap and np.array_equal(la, lo)


def test_no_cpu_fallback(lib, monkeypatch):
    # a missing library must raise, never silently compute on the host
    monkeypatch.setattr(lib, "_lib", None)
    with pytest.raises(ImportError):
        lib.load_library(os.path.join(ROOT, "no_such_libwavelet.so"))


@pytest.mark.parametrize("seed,sigma,hi", [(11, 1 << 19, 7), (12, 300001, 2000)])
def test_library_huffman_large_alphabet_matches_oracle(lib, seed, sigma, hi):
    """Alphabets large enough for the length computation's counting sort to
    split its symbols over several threads, with many equal weights: the
    order of equal weights, and so every length, stays the definition's."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = rng.integers(0, hi + 1, size=sigma).astype(np.uint64)
    hist[rng.integers(0, sigma, size=50)] = rng.integers(1 << 16, 1 << 20, size=50).astype(np.uint64)
    la, ma = lib.huffman_lengths(hist, 32)
    lo, mo = oracle.huffman_lengths(hist, 32)
    assert ma == mo and np.array_equal(la, lo)


@pytest.mark.parametrize("seed,sigma,hi", [(7, 1000, 3), (8, 4096, 1), (9, 300, 40), (10, 70000, 5)])
def test_library_huffman_ties_match_oracle(lib, seed, sigma, hi):
    """Many equal weights (and zero counts): the library's merge order must
    break every tie as the (weight, id) heap of the definition does."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = rng.integers(0, hi + 1, size=sigma).astype(np.uint64)
    la, ma = lib.huffman_lengths(hist, 32)
    lo, mo = oracle.huffman_lengths(hist, 32)
    assert ma == mo and np.array_equal(la, lo)
    assert np.array_equal(lib.canonical_codes(la), oracle.canonical_codes(lo))


def test_unsupported_options_are_rejected_before_device_work(lib):
    # options are checked before any allocation or launch, so this runs on
    # the host alone: an empty sequence with each unsupported option
    so = lib.load_library()
    bad = [dict(tau=9, status=1), dict(tile_symbols=100, status=6), dict(tile_symbols=1000, status=6),
           dict(tile_symbols=16384, status=6), dict(k_chunks=5, status=6),
           dict(select_sample=1000, status=6)]
    # tiles of 2048 and 8192 symbols are for the wavelet matrix only
    tree_bad = [dict(tile_symbols=2048, status=6), dict(tile_symbols=8192, status=6)]
    for b in bad + tree_bad:
        o = lib.BuildOpts()
        for f in ("tau", "tile_symbols", "k_chunks", "select_sample"):
            setattr(o, f, b.get(f, 0))
        h = ctypes.c_void_p()
        fns = [so.wt_build] if b in tree_bad else [so.wm_build, so.wt_build]
        for fn in fns:
            assert fn(None, 0, 4, 2, ctypes.byref(o), None, ctypes.byref(h)) == b["status"], b
            assert not h.value
        if b in tree_bad:
            assert so.multiary_build(None, 0, 4, 2, 4, ctypes.byref(o), None,
                                     ctypes.byref(h)) == b["status"]
            assert so.huff_wt_build(None, 0, 4, 2, None, ctypes.byref(o), None,
                                    ctypes.byref(h)) == b["status"]
    # invalid widths and sigma are rejected the same way
    h = ctypes.c_void_p()
    assert so.wm_build(None, 0, 4, 3, None, None, ctypes.byref(h)) == 1
    assert so.wm_build(None, 0, 0, 2, None, None, ctypes.byref(h)) == 1
    assert so.wm_build(None, 5, 4, 2, None, None, ctypes.byref(h)) == 1
    # the host-memory build checks the same before its copy is enqueued
    for b in bad:
        o = lib.BuildOpts()
        for f in ("tau", "tile_symbols", "k_chunks", "select_sample"):
            setattr(o, f, b.get(f, 0))
        assert so.wm_build_host(None, 0, 4, 2, ctypes.byref(o), None, ctypes.byref(h)) == b["status"], b
        assert not h.value
    assert so.wm_build_host(None, 0, 4, 3, None, None, ctypes.byref(h)) == 1
    assert so.wm_build_host(None, 0, 0, 2, None, None, ctypes.byref(h)) == 1
    assert so.wm_build_host(None, 5, 4, 2, None, None, ctypes.byref(h)) == 1
    assert so.wm_build_host(None, 0, 4, 2, None, None, None) == 1
    # the binding refuses a length beyond the host array before any call
    with pytest.raises(ValueError):
        lib.wm_build_host(np.zeros(4, dtype=np.uint16), 10, n=5)


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_c_client_compiles_and_links(lib, tmp_path, compiler, std):
    # the boundary is plain C: a C99 (and a C++) program using only the
    # header and the CUDA runtime compiles warning-free and links against the
    # library, every call it makes resolving (it is not run without a GPU)
    import shutil
    import subprocess
    cc = shutil.which(compiler)
    if cc is None:
        pytest.skip(f"{compiler} not found")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if not os.path.exists(os.path.join(cuda, "include", "cuda_runtime_api.h")):
        pytest.skip("CUDA headers not found")
    src = os.path.join(ROOT, "tests", "abi_client.c")
    libdir = os.path.dirname(lib.LIB_PATH)
    cmd = [cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic"]
    if compiler == "g++":
        cmd += ["-x", "c++"]
    cmd += [src, "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(cuda, "include"),
            "-o", str(tmp_path / "abi_client"), "-L", libdir, "-l:" + os.path.basename(lib.LIB_PATH),
            "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_huffman_cap_feasibility(lib):
    # 2^cap codewords at most: exactly 2^cap symbols fit (all of length cap);
    # one more symbol has no code, reported as 0 with every length 0
    hist = np.array([1, 2, 3, 4, 5, 6, 7, 1000], dtype=np.uint64)
    la, ma = lib.huffman_lengths(hist, 3)
    assert ma == 3 and np.array_equal(la, np.full(8, 3, np.uint8))
    lo, mo = oracle.huffman_lengths(hist, 3)
    assert mo == 3 and np.array_equal(la, lo)
    la, ma = lib.huffman_lengths(np.append(hist, np.uint64(9)), 3)
    assert ma == 0 and not la.any()
    la, ma = lib.huffman_lengths(np.zeros(5, np.uint64), 3)
    assert ma == 0 and not la.any()


@pytest.mark.parametrize("kind", ["powers", "steep", "noisy"])
def test_library_length_limited_cost_is_optimal(lib, kind):
    """The library's length-limited lengths, pinned without the oracle's
    package-merge: for caps that bind, the cost sum(w * len) equals the
    optimum of an independent dynamic program over depths, every length is
    at most the cap and the code is complete (Kraft sum exactly 1)."""
    from test_oracle_pins import limited_cost_dp
    rng = np.random.default_rng({"powers": 1, "steep": 2, "noisy": 3}[kind])
    if kind == "powers":
        w = [2 ** i for i in range(26)]
    elif kind == "steep":
        w = [int(1.8 ** i) + i for i in range(28)]
    else:
        w = [int(2.1 ** i * rng.uniform(0.6, 1.4)) + 1 for i in range(24)] + [1, 1, 2, 3]
    order = rng.permutation(len(w))
    hist = np.array([w[i] for i in order], dtype=np.uint64)
    _, free_max = lib.huffman_lengths(hist, 64)
    for cap in (free_max - 1, 16, 10, 6):
        if (1 << cap) < len(w):
            continue
        assert cap < free_max  # the cap binds
        ln, mx = lib.huffman_lengths(hist, cap)
        assert 0 < mx <= cap and int(ln.max()) == mx
        assert sum(2.0 ** -int(x) for x in ln) == 1.0
        assert int((hist * ln.astype(np.uint64)).sum()) == limited_cost_dp([int(x) for x in hist],
                                                                          cap)


def test_library_huffman_rejects_out_of_range(lib):
    hist = np.ones(4, dtype=np.uint64)
    ln = np.full(4, 7, dtype=np.uint8)
    so = lib.load_library()
    assert so.wt_huffman_lengths(hist.ctypes.data, (1 << 24) + 1, 32, ln.ctypes.data) == 0
    assert so.wt_huffman_lengths(hist.ctypes.data, 4, 0, ln.ctypes.data) == 0
    assert so.wt_huffman_lengths(hist.ctypes.data, 4, 65, ln.ctypes.data) == 0
    assert (ln == 7).all()  # not written
