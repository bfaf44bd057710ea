#!/usr/bin/env python3
"""Benchmark of the wavelet-matrix build on GB300.

Workload: wavelet matrix of n = 2^30 uint16 symbols over sigma = 2^16 (16
levels), Zipf(s=1.1) over a seeded permutation of the alphabet, plus the rank
directory (2048/512-bit) and select samples (every 4096th one and zero) on
every level.  One step = one complete build (histogram/validation, plan, the
partition passes, bitmaps, zero counts, directories, select samples).

Metric: Gsymbol-levels/s = n * L / step time.  Inputs are resident in HBM for
the device-timed value (2 GiB input > 129 MB L2, so no L2 flush is needed);
``e2e`` repeats the step through the C ABI with the input copied from pinned
host memory and the zero counts read back, inside the timed region.

--impl reference times the CPU oracle (the only reference this project has)
on a bounded sample of the same workload.  Under torchrun every rank builds
its own replica (independent problems, weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gsymbol-levels/s (WM build n=2^30) & %HBM roofline; batched vs plain; query p99"
UNIT = "Gsymbol-levels/s"
SEED = 0x16100352400 + 2
SIGMA = 1 << 16
ZIPF_S = 1.1
PROFILE_TXT = os.path.join(ROOT, "profiles", "k_pass_wm_n2^30_u16_sigma2^16.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--log2n", type=int, default=30, help="sequence length 2^k (default 30)")
    ap.add_argument("--cpu-log2n", type=int, default=24, help="oracle sample length 2^k")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(n_log2):
    return {"workload": f"wavelet matrix build n=2^{n_log2} uint16 sigma=2^16 (16 levels) "
                        "Zipf(1.1) + rank directories + select samples",
            "n": 1 << n_log2, "sigma": SIGMA, "levels": 16, "width_bytes": 2, "tau": 8,
            "tile_symbols": 8192, "l2": "inputs (2 GiB) larger than L2; no flush needed",
            "seed": SEED}


# --------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("k_pass.cuh", "wt_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1610_03524_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """Per-launch DRAM bytes of the pass kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    try:
        txt = open(PROFILE_TXT).read()
    except OSError:
        return None
    kh = ts = None
    for ln in txt.splitlines():
        if ln.startswith("kernel_source_sha256_16:"):
            kh = ln.split(":", 1)[1].strip()
        if ln.startswith("traffic_bytes_per_launch_full_size:"):
            try:
                ts = float(ln.split(":", 1)[1].strip())
            except ValueError:
                ts = None
    return ts if (kh == kernel_hash() and ts) else None


# --------------------------------------------------------------------------
# CPU oracle baseline (test infrastructure, timed as it stands)
# --------------------------------------------------------------------------
def oracle_step(S_sample, sigma):
    import oracle
    import numpy as np
    n = S_sample.size
    t0 = time.perf_counter()
    bits, zeros = oracle.wm_build(S_sample, sigma)
    for l in range(bits.shape[0]):
        oracle.rank_dir(bits[l], n)
        oracle.select_samples(bits[l], n, 0)
        oracle.select_samples(bits[l], n, 1)
    dt = time.perf_counter() - t0
    del np
    return dt


def cpu_baseline(log2n_sample):
    import synth
    n = 1 << log2n_sample
    S = synth.zipf(SEED, n, SIGMA, ZIPF_S, 2)
    dt = oracle_step(S, SIGMA)
    return {"value": n * 16 / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^{log2n_sample} symbols of the workload's distribution (same seed); "
                      f"single-threaded C oracle: WM levels + rank directory + select samples; "
                      f"{dt:.2f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    n = 1 << args.cpu_log2n
    S = synth.zipf(SEED, n, SIGMA, ZIPF_S, 2)
    for _ in range(args.warmup):
        oracle_step(S, SIGMA)
    times = [oracle_step(S, SIGMA) for _ in range(args.steps)]
    tot = sum(times)
    val = n * 16 * args.steps / tot / 1e9
    cfg = workload_config(args.log2n)
    cfg["reference_sample"] = f"2^{args.cpu_log2n} symbols per step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"2^{args.cpu_log2n} symbols of the workload per step, "
                                       "single-threaded C oracle (WM + directories + samples)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# native arm
# --------------------------------------------------------------------------
def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03524_gb300 as wt
    import synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 1 << args.log2n
    L = 16

    # pinned host input, seeded per rank (independent replicas)
    pin = torch.empty(n, dtype=torch.int16).pin_memory()
    synth.zipf(SEED + rank, n, SIGMA, ZIPF_S, 2, addr=pin.data_ptr())
    d = pin.to(dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()

    # warm-up (also builds the pool and the kernel attributes)
    for _ in range(args.warmup):
        h = wt.wm_build(d, SIGMA)
        h.sync()
        h.free()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    handles = []
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    wt.prof_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        handles.append(wt.wm_build(d, SIGMA))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches, pass_launches, pass_ms = wt.prof_read()
    wt.prof_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    for h in handles:
        h.sync()
    handles[0].export()  # completes without error
    for h in handles:
        h.free()
    handles.clear()

    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = ws * n * L / (ms_max * 1e-3) / 1e9

    # roofline of the partition-pass kernel: algorithmic bytes per launch
    # pass 0: read 2 B + write 1 B (next sequence, 8 bits left) + 8 levels/8 B
    # pass 1: read 1 B + 8 levels/8 B
    alg_bytes = args.steps * (4 * n + 2 * n)
    achieved = alg_bytes / (pass_ms * 1e-3) / 1e9 if pass_ms > 0 else None
    peak, peak_kind = measured_peak_hbm()
    traffic = profiled_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic, "kernel": "k_pass (level-group partition pass)",
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6800 GB/s",
            "algorithmic_bytes_per_launch": alg_bytes / max(pass_launches, 1),
            "avg_launch_ms": pass_ms / max(pass_launches, 1),
            "pass_share_of_step": (pass_ms / args.steps) / ms if ms > 0 else None,
            "whole_step_frac_of_Bmin": None}
    # whole-step model B(tau=8) ~ 10.16 n bytes (histogram 2n, passes 6n, directory 2.16n)
    roof["whole_step_frac_of_B_tau8"] = (10.16 * n / (ms * 1e-3) / 1e9) / peak

    # end to end through the C ABI: pinned host input -> device, build, zero counts back
    e2e = None
    if not args.no_e2e:
        dbuf = torch.empty_like(d)
        hz = torch.empty(L, dtype=torch.int64).pin_memory()
        k = max(1, min(args.steps, 5))
        barrier()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        hs = []
        lib = wt.load_library()
        view = wt.ExportView()
        for _ in range(k):
            dbuf.copy_(pin, non_blocking=True)
            h = wt.wm_build(dbuf, SIGMA)
            hs.append(h)
            # the step's result read on the host: wt_export waits for the
            # build and copies the 16 per-level zero counts device -> host
            wt._check(lib.wt_export(h.raw, ctypes.byref(view)), "wt_export")
            hz.numpy()[:] = np.ctypeslib.as_array(view.zeros, shape=(L,)).view(np.int64)
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = f0.elapsed_time(f1) / k
        for h in hs:
            h.free()
        te = torch.tensor([e_ms], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * n * L / (float(te.item()) * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n, "d2h_bytes_per_step": 8 * L, "steps": k}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_log2n)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
                "config": workload_config(args.log2n), "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "parallelism": f"replicas x{ws} (independent builds, no collective)"}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
