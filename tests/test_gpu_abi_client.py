"""The C ABI from a plain C program: tests/abi_client.c builds a wavelet
matrix through include/wavelet.h alone (device memory from the CUDA
runtime), answers rank queries and checks them against counts on the host."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_builds_and_queries(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03524_gb300 as wt
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.dirname(wt.LIB_PATH)
    exe = str(tmp_path / "abi_client")
    cmd = [cc, "-std=c99", os.path.join(ROOT, "tests", "abi_client.c"),
           "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(cuda, "include"),
           "-o", exe, "-L", libdir, "-l:" + os.path.basename(wt.LIB_PATH),
           "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "abi client ok" in r.stdout, r.stdout + r.stderr
