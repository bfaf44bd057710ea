"""Host-side parts of the benchmark: the guard that drops the committed ncu
figures once the pass kernel's source has changed, and the reference arm's
JSON line (the oracle timed on the host; no GPU)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _profile(tmp_path, h):
    p = tmp_path / "prof.md"
    p.write_text("# title\n\nkernel_source_sha256_16: %s\ntraffic_bytes_per_launch_full_size: 3.5e9\n"
                 "issue_active_frac: 0.5\ninst_per_cycle_per_sm: 2.0\n| a | b |\n" % h)
    return str(p)


def test_profile_figures_need_the_current_kernel_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_TXT", _profile(tmp_path, bench.kernel_hash()))
    f = bench.profiled_fields()
    assert f == {"traffic_bytes_per_launch_full_size": 3.5e9, "issue_active_frac": 0.5,
                 "inst_per_cycle_per_sm": 2.0}
    assert bench.profiled_traffic() == 3.5e9
    # a summary taken on other kernel source gives nothing
    monkeypatch.setattr(bench, "PROFILE_TXT", _profile(tmp_path, "0" * 16))
    assert bench.profiled_fields() == {} and bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "PROFILE_TXT", str(tmp_path / "missing.md"))
    assert bench.profiled_fields() == {}


def test_kernel_hash_covers_the_pass_kernel_sources(tmp_path, monkeypatch):
    import shutil
    src = os.path.join(ROOT, "paper_1610_03524_gb300", "csrc")
    dst = tmp_path / "paper_1610_03524_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("k_pass.cuh", "wt_internal.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    for f in ("k_pass.cuh", "wt_internal.cuh"):
        with open(dst / f, "a") as fh:
            fh.write("\n")
        h1 = bench.kernel_hash()
        assert h1 != h0
        h0 = h1


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--cpu-log2n", "16"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_byte_model():
    """Algorithmic bytes of the headline build (the byte model of the
    benchmark's roofline): tau = 8 moves 4 B and 2 B per symbol in its two
    passes and B(8) = 10.16 n for the whole build; tau = 4 narrows the
    intermediate to 12, 8 and 4 bits."""
    import bench
    n = 1 << 20
    assert bench.pass_bytes(n, 16, 2, 8) == [4 * n, 2 * n]
    assert abs(bench.step_bytes(n, 16, 2, 8) / n - 10.15625) < 1e-9
    assert bench.pass_bytes(n, 16, 2, 4) == [4.5 * n, 3.5 * n, 2.5 * n, 1.5 * n]
    assert bench.pass_bytes(n, 3, 1, 8) == [1 * n + 3 * n / 8]
