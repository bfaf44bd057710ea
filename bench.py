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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--log2n", type=int, default=30, help="sequence length 2^k (default 30)")
    ap.add_argument("--cpu-log2n", type=int, default=24, help="oracle sample length 2^k")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["wm", "batch", "serve", "genome", "huff", "select",
                                           "ddmerge"],
                    default="wm",
                    help="wm: the headline wavelet-matrix build (default); batch: 4096 "
                         "wavelet matrices, batched vs plain launches; serve: Poisson "
                         "builds + query batches through the serving loop; genome: "
                         "binary and 4-ary trees of a 2^32-symbol DNA-like text; huff: "
                         "Huffman-shaped and balanced trees over a 2^20 alphabet; select: "
                         "select queries with the sampled and the constant-time select "
                         "directories")
    ap.add_argument("--lam", type=float, default=20.0, help="serve: builds per second")
    ap.add_argument("--qlam", type=float, default=50.0,
                    help="serve: query batches (2^16 queries) per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--no-batch", action="store_true",
                    help="headline: skip the batched-vs-plain sub-measurement")
    ap.add_argument("--no-serve", action="store_true",
                    help="headline: skip the serving-loop sub-measurement")
    ap.add_argument("--no-tune", action="store_true",
                    help="headline: skip the autotuner (default configuration)")
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
            "tile_symbols": 4096, "l2": "inputs (2 GiB) larger than L2; no flush needed",
            "seed": SEED}


def width_for_bits(b):
    return 1 if b <= 8 else (2 if b <= 16 else 4)


def pass_bytes(n, L, w, tau):
    """Algorithmic bytes of each partition pass of a wavelet-matrix build:
    read its input (w bytes on the first pass, the narrowed intermediate
    after), write the next intermediate (not on the last pass), write t
    levels of n bits."""
    out, a = [], 0
    while a < L:
        t = min(tau, L - a)
        in_w = w if a == 0 else width_for_bits(L - a)
        out_w = width_for_bits(L - a - t) if a + t < L else 0
        out.append(n * (in_w + out_w) + n * t / 8)
        a += t
    return out


def step_bytes(n, L, w, tau):
    """B(tau): the whole build's algorithmic bytes -- validation/histogram
    read, the passes, and the directory pass (read the levels, write 16-byte
    records per 2048 bits and the select samples)."""
    return n * w + sum(pass_bytes(n, L, w, tau)) + L * n / 8 + L * n / 128 + L * n / 512


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
                 "--format=csv,noheader,nounits", "-lms", "50"],
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


def profiled_fields():
    """Machine-readable figures of the committed ncu summary of the pass
    kernel (per-launch DRAM traffic at full size, issue-slot use, IPC), if it
    was taken on the current kernel source (else an empty dict)."""
    try:
        txt = open(PROFILE_TXT).read()
    except OSError:
        return {}
    kh, out = None, {}
    for ln in txt.splitlines():
        key, _, val = ln.partition(":")
        if key == "kernel_source_sha256_16":
            kh = val.strip()
        elif key in ("traffic_bytes_per_launch_full_size", "issue_active_frac", "inst_per_cycle_per_sm"):
            try:
                out[key] = float(val.strip())
            except ValueError:
                pass
    return out if kh == kernel_hash() else {}


def profiled_traffic():
    """Per-launch DRAM bytes of the pass kernel from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    return profiled_fields().get("traffic_bytes_per_launch_full_size")


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
                      f"{dt:.2f} s",
            "parallel": cpu_parallel_baseline(S)}


def cpu_parallel_baseline(S, short_lists=False):
    """The same sample through a multi-threaded CPU construction
    (cpu_baseline/: levelwise stable splits over chunks with prefix-summed
    offsets, or big levels every 4 levels with table-driven short lists in
    between), on every host core; median of three runs."""
    import cpu_baseline as cb
    threads = os.cpu_count() or 1
    cb.wm_build(S[:4096], 16, threads, short_lists=short_lists)  # warm-up: threads, pages
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        cb.wm_build(S, 16, threads, short_lists=short_lists)
        ts.append(time.perf_counter() - t0)
    dt = statistics.median(ts)
    kind = ("multi-threaded CPU build, big levels + packed short lists split by table lookup "
            "(cpu_baseline/)" if short_lists else "multi-threaded CPU build, levelwise splits "
            "(cpu_baseline/)")
    out = {"value": S.size * 16 / dt / 1e9, "unit": UNIT, "cores": threads, "kind": kind,
           "sample": f"the same 2^{int(S.size).bit_length() - 1} symbols; WM levels + rank "
                     f"directory + select samples; {dt:.3f} s"}
    if not short_lists:
        out["short_lists"] = cpu_parallel_baseline(S, short_lists=True)
    return out


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

    # the autotuner's configuration (tau, tile size, CTAs per SM), recorded
    # for every later build with zero options; untimed
    if args.no_tune:
        tuning = wt.wm_tuning(n, SIGMA)
    else:
        tuning = wt.wm_autotune_config(d, SIGMA)
    tau = tuning["tau"]
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
    # an event between consecutive builds gives every step's own time
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    e0, e1 = evs[0], evs[-1]
    e0.record(stream)
    for i in range(args.steps):
        handles.append(wt.wm_build(d, SIGMA))
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches, pass_launches, pass_ms = wt.prof_read()
    wt.prof_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
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
    # (tau = 8: pass 0 reads 2 B, writes 1 B of the next sequence and 8 levels
    # = 1 B; pass 1 reads 1 B and writes 1 B of levels)
    alg_bytes = args.steps * sum(pass_bytes(n, L, 2, tau))
    achieved = alg_bytes / (pass_ms * 1e-3) / 1e9 if pass_ms > 0 else None
    peak, peak_kind = measured_peak_hbm()
    # (the committed figure is per launch at n = 2^30: scaled to this n, as
    # a tile's traffic is its own data and two table rows)
    traffic = profiled_traffic()
    if traffic is not None and tau == 8:
        traffic = traffic * n / float(1 << 30)
    elif traffic is not None:
        traffic = None  # taken at tau = 8 only
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic, "kernel": "k_pass (level-group partition pass)",
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6800 GB/s",
            "algorithmic_bytes_per_launch": alg_bytes / max(pass_launches, 1),
            "avg_launch_ms": pass_ms / max(pass_launches, 1),
            "pass_share_of_step": (pass_ms / args.steps) / ms if ms > 0 else None}
    # what bounds the kernel in practice: instruction issue (from the same
    # ncu summary; a diagnostic beside the HBM roofline, 4 issue slots per SM
    # and cycle)
    pf = profiled_fields()
    if "issue_active_frac" in pf:
        roof["issue_diagnostic"] = {"issue_slots_used_frac": pf["issue_active_frac"],
                                    "inst_per_cycle_per_sm": pf.get("inst_per_cycle_per_sm"),
                                    "peak_inst_per_cycle_per_sm": 4.0,
                                    "source": "ncu --set full, 2^26 symbols (profiles/)"}
    # whole-step byte models: B(tau) (tau = 8: ~10.16 n = histogram 2n,
    # passes 6n, directory 2.16n); B_min = n w + L n / 8 + directory writes
    # (L n / 128 + L n / 512 select samples) = 4.156 n, a single ideal pass
    roof["whole_step_frac_of_B_tau"] = (step_bytes(n, L, 2, tau) / (ms * 1e-3) / 1e9) / peak
    roof["whole_step_frac_of_Bmin"] = ((2 + 2 + 16 / 128 + 16 / 512) * n / (ms * 1e-3) / 1e9) / peak

    # end to end through the C ABI with host memory: every step hands the
    # pinned host sequence to wm_build_host (the library copies it in on its
    # host-copy stream and builds on the step's stream) and reads the
    # structure's zero counts back on the host.  Three build streams taken in
    # turn; the host reads step i - 2's result after queueing step i (its
    # release synchronises only step i - 2's stream), so the copies of later
    # steps run while earlier steps build and the GPU never waits for the
    # host between builds
    e2e = None
    if not args.no_e2e:
        hz = torch.empty(L, dtype=torch.int64).pin_memory()
        k = max(1, args.steps)
        sbs = [torch.cuda.Stream() for _ in range(3)]
        lib = wt.load_library()
        view = wt.ExportView()
        ev = lambda: torch.cuda.Event(enable_timing=True)

        def finish(h):
            # the step's result read on the host: wt_export waits for the
            # build (its own stream only) and copies the 16 per-level zero
            # counts device -> host; then the structure is released (its
            # memory returns to the pool)
            wt._check(lib.wt_export(h.raw, ctypes.byref(view)), "wt_export")
            hz.numpy()[:] = np.ctypeslib.as_array(view.zeros, shape=(L,)).view(np.int64)
            h.free()

        def pipeline(k):
            """k steps; returns the first event and each step's events on its
            stream (before the call, and after its build)"""
            f0 = ev()
            f0.record(sbs[0])
            for x in sbs[1:]:
                x.wait_stream(sbs[0])
            bs, be = [ev() for _ in range(k)], [ev() for _ in range(k)]
            pend = []
            for i in range(k):
                s = sbs[i % 3]
                bs[i].record(s)
                pend.append(wt.wm_build_host(pin, SIGMA, stream=s))
                be[i].record(s)
                if len(pend) > 2:
                    finish(pend.pop(0))
            for h in pend:
                finish(h)
            for x in sbs[1:]:
                sbs[0].wait_stream(x)
            return f0, bs, be

        # the same pipeline untimed first (W steps), so that first uses of
        # the pool's memory and of the copy path fall outside the timed steps
        pipeline(max(args.warmup, 3))
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        f0, bs, be = pipeline(k)
        f1 = ev()
        f1.record(sbs[0])
        torch.cuda.synchronize()
        barrier()
        e_ms = f0.elapsed_time(f1) / k
        te = torch.tensor([e_ms], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        # a step's time on its stream: from the end of the build three steps
        # earlier (or the start) through its copy and build
        sms = [bs[i].elapsed_time(be[i]) for i in range(k)]
        e2e = {"value": ws * n * L / (float(te.item()) * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n, "d2h_bytes_per_step": 8 * L, "steps": k,
               "ms_per_step": e_ms,
               "api": "wm_build_host (host sequence in) + wt_export (zero counts out)",
               "timeline": {"stream_ms": [round(x, 3) for x in sms],
                            "stream_ms_median": statistics.median(sms),
                            "exposed_ms_per_step": e_ms - ms}}

    # the batched and the serving workloads, bounded, beside the headline
    # (rank 0 at one GPU; --workload batch / serve run them in full)
    batch = serve = None
    if ws == 1 and not (args.no_batch and args.no_serve):
        pinb, offs, ln, sig, zf, total = _batch_workload()
        if not args.no_batch:
            batch = batch_measure(wt, pinb, offs, ln, sig, total, reps=3, e2e_steps=4)
        if not args.no_serve:
            serve = serve_measure(wt, pinb, offs, ln, sig, lam=20.0, qlam=50.0, duration=3.0,
                                  with_cpu=False)
        del pinb

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.cpu_log2n)

    if rank == 0:
        cfg = workload_config(args.log2n)
        cfg["tau"] = tau
        cfg["tile_symbols"] = tuning["tile_symbols"]
        cfg["tuning"] = {"tau": tau, "tile_symbols": tuning["tile_symbols"],
                         "ctas_per_sm": tuning["ctas_per_sm"], "k_chunks": tuning["k_chunks"],
                         "source": "default (--no-tune)" if args.no_tune
                         else "wm_autotune_config on this sequence, untimed"}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms),
                            "max": max(step_ms)},
                "config": cfg, "roofline": roof, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "parallelism": f"replicas x{ws} (independent builds, no collective)",
                "batch": batch, "serve": serve}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# the other workloads (one JSON line each; not the headline)
# --------------------------------------------------------------------------
def _line(args, metric, value, unit, ms, cfg, **kw):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": kw.pop("n_gpus", 1),
         "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": kw.pop("dtype", "u16"), "data": "synthetic",
         "config": cfg}
    d.update(kw)
    print(json.dumps(d), flush=True)


def _batch_workload(m=4096, world=1, rank=0):
    """The batched configuration: lengths log-uniform in [2^10, 2^24] (total
    capped at 2^31), sigma from {4, 256, 4096, 65536}, uniform or Zipf(1.1),
    uint16; one pinned host array with 16-byte aligned sequence starts.  With
    several ranks, this rank's share of the sequences (independent problems,
    longest-first balanced)."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import synth
    from paper_1610_03524_gb300 import dist as wdist
    ln, sig, zf, sd, total = synth.batch_plan(synth.SEED_BASE + 5, m, 10, 24, 1 << 31)
    if world > 1:
        mine = wdist.shard(ln, world, rank)
        ln, sig, zf, sd = ln[mine], sig[mine], zf[mine], sd[mine]
        m = len(mine)
        total = int(ln.sum())
    offs = np.zeros(m + 1, np.int64)
    for i in range(m):
        offs[i + 1] = offs[i] + (int(ln[i]) + 7) // 8 * 8
    pin = torch.empty(int(offs[-1]), dtype=torch.int16).pin_memory()
    base = pin.data_ptr()

    def gen(i):
        n, s = int(ln[i]), int(sig[i])
        if zf[i]:
            synth.zipf(int(sd[i]), n, s, 1.1, 2, addr=base + 2 * int(offs[i]))
        else:
            synth.uniform(int(sd[i]), n, s, 2, addr=base + 2 * int(offs[i]))

    with ThreadPoolExecutor(8) as ex:
        list(ex.map(gen, range(m)))
    return pin, offs, [int(x) for x in ln], [int(x) for x in sig], zf, int(total)


def batch_measure(wt, pin, offs, ln, sig, total, reps=3, e2e_steps=4):
    """The batched workload at one GPU: one batched build (the batch object,
    wm_batch_build_one) against 4096 plain wm_build calls, wall clock with
    the inputs resident; then end to end through the batch object: each step
    copies the 4 GiB input from pinned host memory, builds the batch and reads
    every sequence's status back, with the next step's copy on a second
    stream overlapping this step's build."""
    import numpy as np
    import torch
    m = len(ln)
    d = pin.to("cuda")
    seqs = [d[int(offs[i]):int(offs[i]) + ln[i]] for i in range(m)]
    items = wt.batch_items(d.data_ptr(), 2 * offs[:m], ln, sig)
    torch.cuda.synchronize()

    def batched():
        b = wt.wm_batch_build_one(items=items)
        st = b.sync()
        assert not st.any(), "batched build failed"
        return b

    def plain():
        hs = [wt.wm_build(seqs[i], sig[i]) for i in range(m)]
        for h in hs:
            h.sync()
        return hs

    def timed(fn, k):
        out = []
        for _ in range(k):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            out.append(time.perf_counter() - t0)
            if isinstance(r, list):
                for h in r:
                    h.free()
            else:
                r.free()
        return out

    timed(batched, 1)
    wt.prof_enable(True)
    tb = timed(batched, reps)
    launches, _, _ = wt.prof_read()
    wt.prof_enable(False)
    b = wt.wm_batch_build_one(items=items)
    b.sync()
    sl = sum(b.handle(i).symbol_levels() for i in range(m))
    b.free()
    timed(plain, 1)
    wt.prof_enable(True)
    tp = timed(plain, 1)
    plain_launches, _, _ = wt.prof_read()
    wt.prof_enable(False)
    mb, mp = statistics.median(tb), statistics.median(tp)
    out = {"workload": "4096 wavelet matrices with directories, lengths log-uniform in "
                       "[2^10, 2^24] (total 2^31 symbols), sigma from {4,256,4096,65536}, "
                       "uniform or Zipf(1.1), uint16",
           "sequences": m, "symbols": int(total), "symbol_levels": int(sl),
           "batched": {"value": sl / mb / 1e9, "unit": UNIT, "ms": 1e3 * mb,
                       "gpu_launches": launches // len(tb), "reps": len(tb)},
           "plain": {"value": sl / mp / 1e9, "unit": UNIT, "ms": 1e3 * mp,
                     "gpu_launches": plain_launches // len(tp), "reps": len(tp)},
           "batched_over_plain": mp / mb,
           "timing": "wall clock around each build (host waits for the results), inputs resident"}
    if e2e_steps:
        dbufs = [torch.empty_like(d), torch.empty_like(d)]
        its = [wt.batch_items(x.data_ptr(), 2 * offs[:m], ln, sig) for x in dbufs]
        sc = torch.cuda.Stream()
        sbs = [torch.cuda.Stream(), torch.cuda.Stream()]
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        built = [torch.cuda.Event(), torch.cuda.Event()]
        torch.cuda.synchronize()

        ev = lambda: torch.cuda.Event(enable_timing=True)

        def pipeline(k):
            # per-step events: the copy on the copy stream, the build on its
            # stream
            cs, ce = [ev() for _ in range(k)], [ev() for _ in range(k)]
            bs, be = [ev() for _ in range(k)], [ev() for _ in range(k)]

            def copy_in(i):
                with torch.cuda.stream(sc):
                    if i >= 2:
                        sc.wait_event(built[i % 2])
                    cs[i].record(sc)
                    dbufs[i % 2].copy_(pin, non_blocking=True)
                    ce[i].record(sc)
                    copied[i % 2].record(sc)

            copy_in(0)
            prev = None
            for i in range(k):
                if i + 1 < k:
                    copy_in(i + 1)
                sbs[i % 2].wait_event(copied[i % 2])
                bs[i].record(sbs[i % 2])
                cur = wt.wm_batch_build_one(items=its[i % 2], stream=sbs[i % 2])
                be[i].record(sbs[i % 2])
                built[i % 2].record(sbs[i % 2])
                if prev is not None:
                    assert not prev.sync().any()
                    prev.free()
                prev = cur
            assert not prev.sync().any()
            prev.free()
            torch.cuda.synchronize()
            return ([round(cs[i].elapsed_time(ce[i]), 3) for i in range(k)],
                    [round(bs[i].elapsed_time(be[i]), 3) for i in range(k)])

        # untimed first (first uses of the buffers and the copy path), then
        # the timed steps
        pipeline(2)
        k = e2e_steps
        t0 = time.perf_counter()
        cms, bms = pipeline(k)
        te = (time.perf_counter() - t0) / k
        out["e2e"] = {"value": sl / te / 1e9, "unit": UNIT, "ms_per_step": 1e3 * te,
                      "h2d_bytes_per_step": int(2 * offs[-1]), "d2h_bytes_per_step": 4 * m,
                      "steps": k, "timeline": {"copy_ms": cms, "build_ms": bms}}
        del dbufs
    del d, seqs
    torch.cuda.empty_cache()
    return out


def serve_measure(wt, pin, offs, ln, sig, lam, qlam, duration, with_cpu=True, seed=None):
    """The serving loop: builds of the batched workload's sequences arriving
    Poisson at lam/s and batches of 2^16 uniform (structure, op, argument)
    queries at qlam/s for `duration` seconds, under a 64 GB admission budget;
    latency from submission to results in host memory."""
    import numpy as np
    host = pin.numpy().view(np.uint16)
    rng = np.random.Generator(np.random.PCG64((synth_seed(5) ^ 0x5e7e) if seed is None else seed))
    srv = wt.Server(budget_bytes=64 << 30)
    D = duration
    tb_arr = np.cumsum(rng.exponential(1.0 / lam, size=int(lam * D * 2) + 10))
    tq_arr = np.cumsum(rng.exponential(1.0 / qlam, size=int(qlam * D * 2) + 10))
    events = sorted([(t, 0) for t in tb_arr if t < D] + [(t, 1) for t in tq_arr if t < D])
    Q = 1 << 16
    # every query batch is drawn before the clock starts: uniform over the
    # builds submitted before it (by submission index), op, and argument
    pre = []
    nsub = 0
    for t, kind in events:
        if kind == 0 and nsub < len(ln):
            nsub += 1
            pre.append(None)
        elif kind == 1 and nsub:
            k = rng.integers(0, nsub, size=Q)
            ns = np.array(ln[:nsub], np.uint64)[k]
            ss = np.array(sig[:nsub], np.uint32)[k]
            op = rng.integers(0, 3, size=Q).astype(np.uint8)
            c = (rng.random(Q) * ss).astype(np.uint32)
            x = (rng.random(Q) * ns).astype(np.uint64)
            x[op == 2] += 1  # select takes k >= 1
            pre.append((k, op, c, x))
        else:
            pre.append(False)
    builds, queries = [], []
    nb = 0
    t0 = time.perf_counter()
    for (t, kind), item in zip(events, pre):
        while time.perf_counter() - t0 < t:
            time.sleep(0.0002)
        if item is None:
            i = nb
            nb += 1
            builds.append(srv.submit_build(host[int(offs[i]):int(offs[i]) + ln[i]], sig[i]))
        elif item:
            k, op, c, x = item
            queries.append(srv.submit_queries(np.array(builds, np.uint64)[k], op, c, x))
    lat_b, lat_q = [], []
    for r in queries:
        st, a, b, _ = srv.poll(r, 0)
        lat_q.append((b - a) * 1e-6)
    for r in builds:
        st, a, b, _ = srv.poll(r)
        lat_b.append((b - a) * 1e-6)
    wall = time.perf_counter() - t0
    srv.close()
    pct = lambda v, p: float(np.percentile(v, p)) if v else None
    out = {"workload": f"serving loop: wavelet-matrix builds of the batched configuration's "
                       f"sequences arriving Poisson at {lam}/s, query batches of 2^16 uniform "
                       f"(structure, op, argument) at {qlam}/s, {D} s of arrivals, 64 GB "
                       f"admission budget",
           "builds": len(builds), "query_batches": len(queries), "queries_per_batch": Q,
           "queries_per_s": len(queries) * Q / wall, "wall_ms": 1e3 * wall,
           "latency_ms": {"query_p50": pct(lat_q, 50), "query_p99": pct(lat_q, 99),
                          "build_p50": pct(lat_b, 50), "build_p99": pct(lat_b, 99)}}
    if with_cpu:
        # the oracle answering queries of the same mix on one sequence of the
        # median length (each answer by definition over the sequence)
        import oracle
        i = int(np.argsort(np.array(ln))[len(ln) // 2])
        S = host[int(offs[i]):int(offs[i]) + ln[i]]
        qn = 256
        op = rng.integers(0, 3, size=qn).astype(np.uint8)
        c = (rng.random(qn) * sig[i]).astype(np.uint32)
        x = (rng.random(qn) * ln[i]).astype(np.uint64)
        x[op == 2] += 1
        t0c = time.perf_counter()
        oracle.access(S, x[op == 0])
        oracle.rank(S, sig[i], c[op == 1], x[op == 1])
        oracle.select(S, sig[i], c[op == 2], x[op == 2])
        dtc = time.perf_counter() - t0c
        out["cpu_baseline"] = {"value": qn / dtc, "unit": "queries/s", "cores": 1,
                               "kind": "oracle",
                               "sample": f"{qn} queries of the same mix on one sequence of "
                                         f"{ln[i]} symbols (the median length), single-threaded "
                                         f"C oracle; {dtc:.3f} s"}
    return out


def run_batch(args, wt):
    ws, rank, _ = dist_env()
    if ws > 1:
        return run_batch_ranks(args, wt)
    pin, offs, ln, sig, zf, total = _batch_workload()
    sampler = ClockSampler(0)
    sampler.start()
    r = batch_measure(wt, pin, offs, ln, sig, total, reps=max(1, args.steps),
                      e2e_steps=0 if args.no_e2e else max(2, min(args.steps, 6)))
    clocks = sampler.stop()
    cpu = None if args.no_cpu else _cpu_batch(pin, offs, ln, sig)
    cfg = {"workload": r["workload"] + ": one batched build (one batch object) vs 4096 plain "
                                       "builds",
           "sequences": r["sequences"], "symbols": r["symbols"], "symbol_levels": r["symbol_levels"],
           "l2": "inputs (4 GiB) larger than L2; no flush needed",
           "parallelism": "one GPU, no collective"}
    _line(args, "Gsymbol-levels/s batched build (wall clock, inputs resident)",
          r["batched"]["value"], UNIT, r["batched"]["ms"], cfg, plain=r["plain"],
          batched_over_plain=r["batched_over_plain"], gpu_launches=r["batched"]["gpu_launches"],
          clocks=clocks, e2e=r.get("e2e"), cpu_baseline=cpu)


def run_batch_ranks(args, wt):
    """Several ranks: each rank builds its share of the sequences (longest
    first, no data-path collective); the slowest rank's time counts."""
    import torch
    import torch.distributed as tdist
    from paper_1610_03524_gb300 import dist as wdist
    ws, rank, _ = dist_env()
    pin, offs, ln, sig, zf, total = _batch_workload(world=ws, rank=rank)
    m = len(ln)
    d = pin.to("cuda")
    items = wt.batch_items(d.data_ptr(), 2 * offs[:m], ln, sig)
    torch.cuda.synchronize()

    def one():
        tdist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = wt.wm_batch_build_one(items=items)
        assert not b.sync().any()
        dt = wdist.max_over_ranks(time.perf_counter() - t0)
        sl = sum(b.handle(i).symbol_levels() for i in range(m))
        b.free()
        return dt, sl

    for _ in range(args.warmup):
        one()
    ts, sl = [], 0
    for _ in range(max(1, args.steps)):
        dt, sl = one()
        ts.append(dt)
    sl = int(wdist.sum_over_ranks(sl))
    total = int(wdist.sum_over_ranks(total))
    mb = statistics.median(ts)
    if rank != 0:
        return
    cfg = {"workload": "4096 wavelet matrices with directories (batched configuration), "
                       "sequences sharded over ranks", "symbols": total, "symbol_levels": sl,
           "parallelism": f"sequences sharded over {ws} rank(s), no data-path collective"}
    _line(args, "Gsymbol-levels/s batched build (wall clock, inputs resident)", sl / mb / 1e9,
          UNIT, 1e3 * mb, cfg, n_gpus=ws)


def _cpu_batch(pin, offs, ln, sig, target=1 << 24):
    """The oracle on the batch's first sequences (about 2^24 symbols): WM
    levels, rank directory and select samples of every level."""
    import numpy as np
    import oracle
    host = pin.numpy().view(np.uint16)
    tot = sl = 0
    t0 = time.perf_counter()
    i = 0
    while i < len(ln) and tot < target:
        S = host[int(offs[i]):int(offs[i]) + ln[i]]
        bits, _ = oracle.wm_build(S, sig[i])
        for l in range(bits.shape[0]):
            oracle.rank_dir(bits[l], S.size)
            oracle.select_samples(bits[l], S.size, 0)
            oracle.select_samples(bits[l], S.size, 1)
        tot += S.size
        sl += S.size * bits.shape[0]
        i += 1
    dt = time.perf_counter() - t0
    return {"value": sl / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the first {i} sequences of the batch ({tot} symbols), single-threaded C "
                      f"oracle: WM levels + rank directory + select samples; {dt:.2f} s"}


def run_serve(args, wt):
    pin, offs, ln, sig, zf, total = _batch_workload()
    r = serve_measure(wt, pin, offs, ln, sig, args.lam, args.qlam, args.duration,
                      with_cpu=not args.no_cpu)
    cfg = {"workload": r["workload"], "builds": r["builds"], "query_batches": r["query_batches"],
           "queries_per_batch": r["queries_per_batch"]}
    _line(args, "queries/s through the serving loop (arrival -> answers on host)",
          r["queries_per_s"], "queries/s", r["wall_ms"], cfg, cpu_baseline=r.get("cpu_baseline"),
          latency_ms=r["latency_ms"])


def run_select(args, wt):
    """Select queries through the sampled select directory and through the
    constant-time one (FLAG_SELECT_O1), on the headline wavelet matrix
    (n = 2^30, sigma = 2^16) and on a 2^32-bit bitvector whose ones
    alternate between dense stretches and stretches with one 1 in 300 bits
    (long sampled searches); plus what the constant-time directory adds to
    the build."""
    import numpy as np
    import torch
    import synth
    res = {}
    Q = 1 << 22
    rng = np.random.Generator(np.random.PCG64(synth_seed(2) ^ 0x5e1))

    def timed(fn, reps=5):
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[1:])

    # wavelet matrix of the headline workload
    n = 1 << 30
    pin = torch.empty(n, dtype=torch.int16).pin_memory()
    synth.zipf(SEED, n, SIGMA, ZIPF_S, 2, addr=pin.data_ptr())
    d = pin.to("cuda")
    S = pin.numpy().view(np.uint16)
    hist = np.bincount(S, minlength=SIGMA)
    present = np.nonzero(hist)[0]
    c = present[rng.integers(0, present.size, Q)].astype(np.uint32)
    k = (rng.random(Q) * hist[c]).astype(np.uint64) + 1
    dc, dk = torch.from_numpy(c.view(np.int32)).cuda(), torch.from_numpy(k.view(np.int64)).cuda()
    out = torch.empty(Q, dtype=torch.int64, device="cuda")
    for name, fl in (("sampled", 0), ("o1", wt.FLAG_SELECT_O1)):
        bms = timed(lambda: wt.wm_build(d, SIGMA, flags=fl).free(), 3)
        h = wt.wm_build(d, SIGMA, flags=fl)
        h.sync()
        qms = timed(lambda: h.select(dc, dk, out))
        res[f"wm_{name}"] = {"build_ms": bms, "select_ms": qms, "queries_per_s": Q / qms * 1e3}
        h.free()
    del d
    # bitvector with long sparse stretches
    nb = 1 << 32
    words = np.zeros(nb // 64, dtype=np.uint64)
    st = np.arange(nb // (1 << 24))
    dense = st % 2 == 0
    # dense stretches: random words; sparse stretches: one 1 every 300 bits
    wpr = (1 << 24) // 64
    rw = synth.words(synth_seed(2) ^ 0xb17, int(dense.sum()) * wpr)
    for i, s0 in enumerate(np.nonzero(dense)[0]):
        words[s0 * wpr:(s0 + 1) * wpr] = rw[i * wpr:(i + 1) * wpr]
    for s0 in np.nonzero(~dense)[0]:
        ones = np.arange(s0 << 24, (s0 + 1) << 24, 300, dtype=np.uint64)
        np.bitwise_or.at(words, (ones >> np.uint64(6)).astype(np.int64),
                         np.left_shift(np.uint64(1), ones & np.uint64(63)))
    dw = torch.from_numpy(words.view(np.int64)).cuda()
    for name, fl in (("sampled", 0), ("o1", wt.FLAG_SELECT_O1)):
        bms = timed(lambda: wt.rs_build(dw, nb, flags=fl).free(), 3)
        h = wt.rs_build(dw, nb, flags=fl)
        ex_ones = nb - int(h.export().zeros[0])
        k1 = (rng.random(Q) * ex_ones).astype(np.uint64) + 1
        dk1 = torch.from_numpy(k1.view(np.int64)).cuda()
        dc1 = torch.ones(Q, dtype=torch.int32, device="cuda")
        qms = timed(lambda: h.select(dc1, dk1, out))
        res[f"bitvector_{name}"] = {"build_ms": bms, "select_ms": qms,
                                    "queries_per_s": Q / qms * 1e3}
        h.free()
    del dw
    # 4-ary tree of the DNA-like text (n = 2^32, sigma 5): select per digit
    # value on every digit level (generalized select)
    ng = 1 << 32
    gpin = torch.empty(ng, dtype=torch.uint8).pin_memory()
    synth.genome(synth_seed(3), ng, addr=gpin.data_ptr())
    dg = gpin.to("cuda")
    del gpin
    cnt = torch.zeros(5, dtype=torch.int64, device="cuda")
    for o in range(0, ng, 1 << 28):
        cnt += torch.bincount(dg[o:o + (1 << 28)].to(torch.int32), minlength=5)
    cnt = cnt.cpu().numpy()
    presg = np.nonzero(cnt)[0]
    cg = presg[rng.integers(0, presg.size, Q)].astype(np.uint32)
    kg = (rng.random(Q) * cnt[cg]).astype(np.uint64) + 1
    dcg = torch.from_numpy(cg.view(np.int32)).cuda()
    dkg = torch.from_numpy(kg.view(np.int64)).cuda()
    for name, fl in (("sampled", 0), ("o1", wt.FLAG_SELECT_O1)):
        bms = timed(lambda: wt.multiary_build(dg, 5, flags=fl).free(), 3)
        h = wt.multiary_build(dg, 5, flags=fl)
        h.sync()
        qms = timed(lambda: h.select(dcg, dkg, out))
        res[f"multiary_{name}"] = {"build_ms": bms, "select_ms": qms,
                                   "queries_per_s": Q / qms * 1e3}
        h.free()
    del dg
    cpu = None
    if not args.no_cpu:
        import oracle
        Sm = np.ascontiguousarray(S[: 1 << 22])
        hm = np.bincount(Sm, minlength=SIGMA)
        pm = np.nonzero(hm)[0]
        cq = pm[rng.integers(0, pm.size, 256)].astype(np.uint32)
        kq = (rng.random(256) * hm[cq]).astype(np.uint64) + 1
        t0 = time.perf_counter()
        oracle.select(Sm, SIGMA, cq, kq)
        dt = time.perf_counter() - t0
        cpu = {"value": 256 / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"256 selects on the first 2^22 symbols, single-threaded C oracle "
                         f"(scan by definition); {dt:.3f} s"}
    cfg = {"workload": f"2^22 select queries (c, k uniform over present symbols and their "
                       f"counts) on the wavelet matrix of n=2^30 uint16 Zipf(1.1), sigma 2^16; "
                       f"and 2^22 select-1 queries on a 2^32-bit bitvector of dense and 1-in-300 "
                       f"stretches; and 2^22 selects on the 4-ary tree of the n=2^32 DNA-like "
                       f"text (sigma 5); sampled vs constant-time select directory",
           "queries": Q}
    _line(args, "select queries/s, constant-time directory (wavelet matrix n=2^30)",
          res["wm_o1"]["queries_per_s"], "queries/s", res["wm_o1"]["select_ms"], cfg, dtype="u16",
          results=res, cpu_baseline=cpu)


def run_ddmerge(args, wt):
    """Domain decomposition (Section 4.2) of the headline sequence: the
    wavelet matrix of n = 2^30 uint16 Zipf(1.1) over 2^16 built as 8
    consecutive pieces and merged, against one build of the whole.  The merge
    reads every piece's bits and writes the whole's once: 2 n L / 8 bytes."""
    import numpy as np
    import torch
    import synth
    n, R = 1 << args.log2n, 8
    L = 16
    pin = torch.empty(n, dtype=torch.int16).pin_memory()
    synth.zipf(SEED, n, SIGMA, ZIPF_S, 2, addr=pin.data_ptr())
    d = pin.to("cuda")
    del pin
    cut = [i * n // R for i in range(R + 1)]
    pieces_t = [d[a:b] for a, b in zip(cut[:-1], cut[1:])]

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts[args.warmup:]) if len(ts) > args.warmup else ts[-1]

    reps = args.warmup + args.steps
    single = timed(lambda: wt.wm_build(d, SIGMA).free(), reps)

    def build_pieces():
        return [wt.wm_build(x, SIGMA) for x in pieces_t]

    piece_ms = timed(lambda: [h.free() for h in build_pieces()], reps)
    parts = build_pieces()
    for h in parts:
        h.sync()
    merge_nodir = timed(lambda: wt.dd_merge(parts, flags=wt.FLAG_NO_DIRECTORY).free(), reps)
    merge_ms = timed(lambda: wt.dd_merge(parts).free(), reps)
    for h in parts:
        h.free()
    alg = 2 * n * L / 8
    peak, peak_kind = measured_peak_hbm()
    ach = alg / (merge_nodir * 1e-3) / 1e9
    tot = piece_ms + merge_ms
    cfg = {"workload": f"wavelet matrix of n=2^{args.log2n} uint16 Zipf(1.1) sigma=2^16 as {R} "
                       f"pieces built apart and merged (domain decomposition), vs one build",
           "pieces": R, "l2": "inputs larger than L2; no flush needed"}
    _line(args, "Gsymbol-levels/s (pieces + merge, with directories)", n * L / tot / 1e6,
          "Gsymbol-levels/s", tot, cfg,
          results={"single_build_ms": single, "pieces_build_ms": piece_ms,
                   "merge_ms_with_directories": merge_ms, "merge_ms_bits_only": merge_nodir},
          roofline={"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": None,
                    "kernel": "wt_dd_merge without directories (node sizes, plan, k_dd_copy)",
                    "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                    if peak_kind == "measured" else "fallback",
                    "algorithmic_bytes_per_launch": alg})


def synth_seed(k):
    import synth
    return synth.SEED_BASE + k


def run_tree(args, wt):
    """genome: binary WT and 4-ary WT of n = 2^32 uint8 over {A,C,G,T} plus a
    sentinel (sigma 5); huff: Huffman-shaped and balanced WT of n = 2^28 uint32
    Zipf(1.0) over 2^20 symbols."""
    import numpy as np
    import torch
    import synth
    if args.workload == "genome":
        n = 1 << 32
        pin = torch.empty(n, dtype=torch.uint8).pin_memory()
        synth.genome(synth_seed(3), n, addr=pin.data_ptr())
        sigma, builds = 5, [("wt", wt.wt_build), ("multiary", wt.multiary_build)]
        desc = "n=2^32 uint8 DNA-like text (order-3 chain, bursts, sentinel), sigma=5"
    else:
        n = 1 << 28
        pin = torch.empty(n, dtype=torch.int32).pin_memory()
        synth.zipf(synth_seed(4), n, 1 << 20, 1.0, 4, addr=pin.data_ptr())
        sigma, builds = 1 << 20, [("huffman", wt.huff_wt_build), ("wt", wt.wt_build)]
        desc = "n=2^28 uint32 Zipf(1.0) over 2^20 symbols"
    d = pin.to("cuda")
    torch.cuda.synchronize()
    res = {}
    for name, fn in builds:
        for _ in range(args.warmup):
            h = fn(d, sigma)
            h.sync()
            h.free()
        # wall clock over K builds with two in flight (the Huffman build
        # finishes from a library thread, so the host's code construction of
        # one build overlaps the device work of the previous one); each
        # build is complete (synchronised) before the clock stops
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h = fn(d, sigma)
        h.sync()
        single = time.perf_counter() - t1
        sl = h.symbol_levels()
        h.free()
        wt.prof_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = None
        for _ in range(args.steps):
            h = fn(d, sigma)
            if prev is not None:
                prev.sync()
                prev.free()
            prev = h
        prev.sync()
        prev.free()
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0) / args.steps
        la, pl, pms = wt.prof_read()
        wt.prof_enable(False)
        res[name] = {"ms_per_build": ms, "symbol_levels": sl, "gsl_per_s": sl / ms / 1e6,
                     "pass_ms": pms / args.steps, "gpu_launches": la // args.steps,
                     "single_build_ms": 1e3 * single,
                     "timing": "wall clock, two builds in flight, each synchronised"}
    cpu = None
    if not args.no_cpu:
        cpu = _cpu_tree(args.workload, pin.numpy(), sigma)
    first = builds[0][0]
    cfg = {"workload": f"{' and '.join(b[0] for b in builds)} wavelet trees with directories, "
                       f"{desc}", "n": n, "sigma": sigma}
    _line(args, f"Gsymbol-levels/s ({first} build)", res[first]["gsl_per_s"], UNIT,
          res[first]["ms_per_build"], cfg, dtype="u8" if args.workload == "genome" else "u32",
          builds=res, gpu_launches=res[first]["gpu_launches"], cpu_baseline=cpu)


def _cpu_tree(workload, host, sigma):
    """The oracle on a prefix of the same input: the first build of the line
    (balanced WT for the genome, Huffman-shaped WT for the 2^20 alphabet)
    with the directories of every level."""
    import numpy as np
    import oracle
    n = 1 << 24 if workload == "genome" else 1 << 22
    S = np.ascontiguousarray(host[:n])
    t0 = time.perf_counter()
    if workload == "genome":
        bits = oracle.wt_build(S, sigma)
        for l in range(bits.shape[0]):
            oracle.rank_dir(bits[l], n)
            oracle.select_samples(bits[l], n, 0)
            oracle.select_samples(bits[l], n, 1)
        sl = n * bits.shape[0]
        what = "balanced WT levels + rank directory + select samples"
    else:
        hist = np.bincount(S.astype(np.int64), minlength=sigma).astype(np.uint64)
        ln, _ = oracle.huffman_lengths(hist, 32)
        cd = oracle.canonical_codes(ln)
        bits, woff, nl = oracle.huff_wt_build(S, ln, cd)
        for l in range(nl.size):
            lv = bits[int(woff[l]):int(woff[l + 1])]
            oracle.rank_dir(lv, int(nl[l]))
        sl = int(nl.sum())
        what = "Huffman code + Huffman-shaped WT levels + rank directory"
    dt = time.perf_counter() - t0
    return {"value": sl / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first 2^{n.bit_length() - 1} symbols of the input, single-threaded C oracle: "
                      f"{what}; {dt:.2f} s"}


def run_other(args):
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle arm is timed on the headline workload only"}))
        return 0
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_03524_gb300 as wt
    torch.cuda.set_device(local)
    if args.workload == "batch":
        if ws > 1:
            import torch.distributed as tdist
            tdist.init_process_group("nccl")
        run_batch(args, wt)
        if ws > 1:
            tdist.barrier()
            tdist.destroy_process_group()
        return 0
    if rank != 0:
        return 0  # the other workloads run on one GPU
    if args.workload == "batch":
        run_batch(args, wt)
    elif args.workload == "serve":
        run_serve(args, wt)
    elif args.workload == "select":
        run_select(args, wt)
    elif args.workload == "ddmerge":
        run_ddmerge(args, wt)
    else:
        run_tree(args, wt)
    return 0


def main():
    args = parse()
    if args.workload != "wm":
        return run_other(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
