#!/usr/bin/env python
"""Benchmark: Gsamples/s of the modified-ziggurat generator on GB300.

A step is one pass of the hot path (layer index, fast path, fringe) over one
batch: n = 2^28 standard normals in FP64 (2 GiB, larger than the 129 MB L2,
so no flush is needed), each step on fresh counters.  One JSON line on
rank 0.  `--impl reference` times the CPU oracle on the host cores instead
(rank 0 only).  Multi-GPU: one process per GPU under torchrun, each rank on
its own counter range (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_1403_6870_gb300.shard import step_counter  # noqa: E402

METRIC = "Gsamples/s (exp & normal, FP64/FP32) and % HBM-write roofline; batched vs plain"
UNIT = "Gsamples/s"
DEFAULT_WORKLOAD = "normal_f64_2p28"
KERNEL_SRCS = [os.path.join(ROOT, "paper_1403_6870_gb300", "csrc", f)
               for f in ("zig_gen.cu", "zig_device.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "gen_kernel_normal_f64_traffic.txt")
PIPES_FILE = os.path.join(ROOT, "profiles", "gen_kernel_moments_f32_pipes.txt")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="zig", choices=["zig", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(W.WORKLOADS))
    p.add_argument("--n", type=int, default=None,
                   help="override the per-step size (for small profiling captures)")
    p.add_argument("--keying", default="index", choices=["index", "packed"],
                   help="uniform keying: per-index (the default, zig_exponential/zig_normal) "
                        "or the opt-in packed keying (zig_generate ZIG_KEY_PACKED)")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the launch-shape autotuner (use the default shape)")
    p.add_argument("--batch-requests", type=int, default=None,
                   help="time only zig_batch on the first K requests of the serving mix "
                        "(a small case for profiling) and print its line")
    p.add_argument("--clock-soak", type=float, default=1.0,
                   help="seconds of untimed launches run under the clock sampler just before "
                        "the timed region (0 for profiling commands)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the CPU baseline, e2e, variant and batch measurements")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash() -> str:
    """First 16 hex digits of the SHA-256 of the generation kernel's device
    sources: zig_gen.cu up to its host-side section, then zig_device.cuh."""
    h = hashlib.sha256()
    for path in KERNEL_SRCS:
        with open(path, "rb") as f:
            data = f.read()
        cut = data.find(b"\n// Host side\n")
        h.update(data if cut < 0 else data[:cut])
    return h.hexdigest()[:16]


def recorded_traffic(n: int):
    """DRAM bytes (read + write) of one launch of n samples from the
    committed ncu summary, or None if it was taken for another n or the
    kernel source changed since."""
    try:
        kv = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_hash():
            return None
        if int(kv["n_captured"]) != n:
            return None
        return float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])
    except Exception:
        return None


def recorded_pipes(keying: str):
    """ncu pipe utilisation of the fused-reduction kernel (FP32 normals) for
    a keying ("index" or "packed") from the committed summary, or None if
    the kernel source changed since it was taken.  Lines `<keying>.<key>:
    value` hold the busy percentages of the integer multiply pipe
    (fmaheavy), the ALU pipe and instruction issue."""
    try:
        kv = {}
        with open(PIPES_FILE) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha256_16") != kernel_hash():
            return None
        pipes = {name: float(kv[f"{keying}.{name}_pct"]) for name in ("fmaheavy", "alu", "issue")}
        bound = max(pipes, key=pipes.get)
        return {"bound": "alu", "pipe": bound, "achieved": pipes[bound], "peak": 100.0,
                "unit": "% busy (ncu, of the pipe's peak)", "frac": pipes[bound] / 100.0,
                "pipes_pct": pipes, "traffic": None,
                "source": os.path.relpath(PIPES_FILE, ROOT) + f" (n = {kv['n_captured']})"}
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.tmp, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        with open(self.tmp.name) as f:
            rows = [r.split(",") for r in f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def soak(step, first: int, ms_per_step: float, stream, seconds: float):
    """Untimed steps for about `seconds`, run just before the timed region
    with the clock sampler already running, so that it sees the same
    launches under load even when K steps last only milliseconds.  Returns
    the number of steps run (their counters follow `first`)."""
    import torch

    count = int(seconds * 1e3 / max(ms_per_step, 1e-3)) if seconds > 0 else 0
    for k in range(count):
        step(first + k)
    torch.cuda.synchronize()
    return count


def oracle_rate(dist: int, dtype: int, offset: int, n: int, nthreads=None):
    """Oracle throughput (samples/s) on nthreads host cores (default: all)
    for n counters."""
    from oracle import oracle

    oracle.build()
    oracle.tables(oracle.EXP)
    oracle.tables(oracle.NORMAL)  # built before the timed region
    threads = nthreads or oracle.default_threads()
    t0 = time.perf_counter()
    oracle.fill(dist, dtype, W.SEED, offset, n, nthreads=threads)
    return n / (time.perf_counter() - t0), threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    c = W.WORKLOADS[args.workload]
    from oracle import oracle

    oracle.build()
    threads = oracle.default_threads()
    # size each step so the whole run takes about a minute
    cal, _ = oracle_rate(c["dist"], c["dtype"], c["offset"], 1 << 20)
    budget = 60.0 / max(1, args.steps + args.warmup)
    per = int(min(max(cal * budget, 1 << 14), 1 << 26))
    per = 1 << int(math.log2(per))
    for k in range(args.warmup):
        oracle.fill(c["dist"], c["dtype"], W.SEED, c["offset"] + k * per, per, nthreads=threads)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.fill(c["dist"], c["dtype"], W.SEED, c["offset"] + (args.warmup + k) * per, per,
                    nthreads=threads)
    dt = time.perf_counter() - t0
    value = per * args.steps / dt / 1e9
    sample = f"{per} counters per step of {args.workload} (fresh counters each step)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if c["dtype"] == W.F64 else "f32", "data": "synthetic",
        "config": {"workload": args.workload, "dist": "normal" if c["dist"] else "exponential",
                   "n_per_step": per, "seed": W.SEED,
                   "note": "the CPU oracle on the host cores (rank 0 only); no GPU work"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_fused(args):
    """The fused workload as the bench line: each step reduces n fresh FP32
    normals to power sums and a histogram (nothing stored)."""
    import torch
    import torch.distributed as dist

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    c = W.WORKLOADS[args.workload]
    n = args.n or c["n"]
    keying = 1 if args.keying == "packed" else 0
    stream = torch.cuda.current_stream()
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    hist = torch.zeros(4098, dtype=torch.int64, device="cuda")
    ws = torch.empty(z.zig_moments_workspace_bytes(c["dist"], c["dtype"]), dtype=torch.uint8,
                     device="cuda")

    def step(k):
        fused_call(z, c["dist"], c["dtype"], keying, n, W.SEED,
                   step_counter(c["offset"], k, rank, world, n), sums, hist, ws, stream)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.warmup):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    est_ms = e0.elapsed_time(e1) / max(1, args.warmup)
    with ClockSampler(local_rank) as clk:
        nsoak = soak(step, args.warmup, est_ms, stream, args.clock_soak)
        first = args.warmup + nsoak
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            step(first + k)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = n * args.steps * world / (ms / 1e3) / 1e9
    peak, mhz = alu_peak(z)
    achieved = n / (ms / args.steps / 1e3) * (0.25 if keying else 1.0) * PHILOX_OPS_PER_BLOCK / 1e12
    # e2e: the same steps with the results (sums, histogram) read to host memory
    hs = torch.empty(4, dtype=torch.float64, pin_memory=True)
    hh = torch.empty(4098, dtype=torch.int64, pin_memory=True)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = args.steps
    if world > 1:
        dist.barrier()
    f0.record(stream)
    for k in range(e2e_steps):
        step(first + args.steps + k)
        hs.copy_(sums, non_blocking=True)
        hh.copy_(hist, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    if world > 1:  # whole-job rate: the slowest rank's time
        t = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (Philox counters; seed 0x0123456789ABCDEF, fresh counters per step)",
        "config": {"workload": args.workload, "dist": "normal", "n_per_step_per_gpu": n,
                   "keying": args.keying, "l2": "nothing is stored; no flush needed",
                   "parallelism": f"counter-range shards x{world}"},
        "clocks": dict(clk.summary(), window=f"{nsoak} untimed steps of the same launch "
                       f"(~{args.clock_soak:g} s) just before the timed region, and the region"),
        "gpu_launches": args.steps,
        "roofline": dict(recorded_pipes(args.keying) or {
            "bound": "alu", "achieved": None, "peak": 100.0, "frac": None, "traffic": None,
            "unit": "% busy (ncu)", "note": "no ncu summary for the current kernel source"},
            kernel="gen_kernel<normal,float,MomentSink>",
            philox={"achieved_tops": achieved, "lane_issue_peak_tops": peak,
                    "peak_source": f"SMs x 4 schedulers x 32 lanes x {mhz:.0f} MHz",
                    "ops_per_launch": n * (0.25 if keying else 1.0) * PHILOX_OPS_PER_BLOCK}),
        "e2e": {"value": n * world * e2e_steps / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": (4 * 8 + 4098 * 8) * world},
        "device_status": z.zig_strerror(z.zig_status_poll(stream)),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_zig(args):
    import torch
    import torch.distributed as dist

    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    c = W.WORKLOADS[args.workload]
    n = args.n or c["n"]
    tdt = torch.float64 if c["dtype"] == W.F64 else torch.float32
    esize = 8 if c["dtype"] == W.F64 else 4
    if args.keying == "packed":
        def fn(out_, n_, seed_, offset_, stream=None):
            z.zig_generate(c["dist"], z.ZIG_KEY_PACKED, out_, n_, seed_, offset_, stream=stream)
    else:
        fn = z.zig_normal if c["dist"] == W.NORMAL else z.zig_exponential
    out = torch.empty(n, dtype=tdt, device="cuda")
    stream = torch.cuda.current_stream()

    def counter(step):  # fresh counters per step and rank (weak scaling)
        return step_counter(c["offset"], step, rank, world, n)

    tuned = None
    if not args.no_tune and args.keying == "index":
        # pick the launch shape on the workload's own output buffer (> L2)
        chosen, results = z.zig_autotune(c["dist"], c["dtype"], out, reps=3, stream=stream)
        tuned = {"chosen": chosen, "measured": results}
    def step(k):
        fn(out, n, W.SEED, counter(k), stream=stream)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.warmup):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    est_ms = e0.elapsed_time(e1) / max(1, args.warmup)
    with ClockSampler(local_rank) as clk:
        nsoak = soak(step, args.warmup, est_ms, stream, args.clock_soak)
        first = args.warmup + nsoak
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(args.steps):
            step(first + k)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    status = z.zig_status_poll(stream)
    value = n * args.steps * world / (ms / 1e3) / 1e9
    launch_ms = ms / args.steps  # one kernel launch per step
    peak, peak_src = measured_peak()
    achieved = n * esize / (launch_ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if c["dtype"] == W.F64 else "f32",
        "data": "synthetic (Philox counters; seed 0x0123456789ABCDEF, fresh counters per step)",
        "config": {"workload": args.workload, "dist": "normal" if c["dist"] else "exponential",
                   "n_per_step_per_gpu": n, "output_bytes": n * esize,
                   "l2": "output {:.2f} GiB per step {} 129 MB L2; no flush".format(
                       n * esize / 2**30, ">" if n * esize > 129e6 else "<="),
                   "parallelism": f"counter-range shards x{world}"},
        "clocks": dict(clk.summary(), window=f"{nsoak} untimed steps of the same launch "
                       f"(~{args.clock_soak:g} s) just before the timed region, and the region"),
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic(n) if (args.keying == "index" and
                                                        args.workload == DEFAULT_WORKLOAD) else None,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, copy)",
                     "kernel": "gen_kernel<{},{}{}>".format(
                         "normal" if c["dist"] else "exp",
                         "double" if c["dtype"] == W.F64 else "float",
                         ",packed" if args.keying == "packed" else ""),
                     "algorithmic_bytes_per_launch": n * esize},
        "device_status": z.zig_strerror(status),
        "launch_shape": z.zig_tune_get(c["dist"], c["dtype"]) if args.keying == "index"
        else "default",
        "keying": args.keying,
    }
    if tuned is not None:
        line["autotune"] = tuned
    if not args.no_extras:
        line["e2e"] = measure_e2e(z, fn, out, n, esize, counter, stream, args)
    if rank == 0 and world == 1 and not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(c)
        line["variants"] = measure_variants(z, stream)
        line["packed_keying"] = measure_packed(z, stream)
        line["i_max_1024"] = measure_i1024(z, stream)
        line["fused"] = measure_fused(z, stream)
        line["precision_f32"] = measure_precision(z, stream)
        del out
        torch.cuda.empty_cache()
        line["batch"] = measure_batch(z, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_e2e(z, fn, out, n, esize, counter, stream, args):
    """Same metric through the public call with the result in host memory
    every step: the call writes a page-locked host buffer directly (its
    device alias; NVLink-C2C on Grace), so each step's n outputs cross to
    the host inside the timed region.  For comparison the same steps are
    also timed writing device memory and copying it to the host buffer.
    With several ranks each region starts after a barrier and its time is
    the maximum over the ranks, so the values are whole-job rates."""
    import torch
    import torch.distributed as dist

    _, world, _ = dist_env()
    host = torch.empty(n, dtype=out.dtype, pin_memory=True)
    steps = args.steps  # as many steps as the device-timed region

    def timed(body):
        for k in range(2):
            body(k)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            body(2 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    ms = timed(lambda k: fn(host, n, W.SEED, counter(k), stream=stream))

    def via_copy(k):
        fn(out, n, W.SEED, counter(k), stream=stream)
        host.copy_(out, non_blocking=True)

    ms_copy = timed(via_copy)
    total = n * world  # outputs of all ranks per step
    return {"value": total * steps / (ms / 1e3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": total * esize, "steps": steps,
            "d2h_gb_s": total * esize * steps / (ms / 1e3) / 1e9,
            "via_device_buffer_and_copy": {
                "value": total * steps / (ms_copy / 1e3) / 1e9,
                "d2h_gb_s": total * esize * steps / (ms_copy / 1e3) / 1e9},
            "note": "inputs are (seed, offset, n) launch arguments; each step the call writes "
                    "its n outputs into page-locked host memory (the result is in host memory "
                    "when the step's work ends)"}


def cpu_baseline(c):
    n, n1 = 1 << 25, 1 << 22
    rate, threads = oracle_rate(c["dist"], c["dtype"], c["offset"], n)
    rate1, _ = oracle_rate(c["dist"], c["dtype"], c["offset"], n1, nthreads=1)
    return {"value": rate / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} counters of the workload, all host cores",
            "single_thread": {"value": rate1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"first {n1} counters of the workload, one thread"}}


def measure_variants(z, stream, steps: int = 100):
    """Throughput of the other dist/dtype combinations (2^28 counters each),
    and of the FP32 pairs at their workload's own launch size, 2^30."""
    import torch

    res = {}
    for name, dist, dtype, n in (("exp_f64", W.EXP, W.F64, 1 << 28),
                                 ("normal_f64", W.NORMAL, W.F64, 1 << 28),
                                 ("exp_f32", W.EXP, W.F32, 1 << 28),
                                 ("normal_f32", W.NORMAL, W.F32, 1 << 28),
                                 ("exp_f32_2p30", W.EXP, W.F32, 1 << 30),
                                 ("normal_f32_2p30", W.NORMAL, W.F32, 1 << 30)):
        tdt = torch.float64 if dtype == W.F64 else torch.float32
        es = 8 if dtype == W.F64 else 4
        buf = torch.empty(n, dtype=tdt, device="cuda")
        fn = z.zig_normal if dist == W.NORMAL else z.zig_exponential
        chosen, _ = z.zig_autotune(dist, dtype, buf, reps=3, stream=stream)
        for k in range(5):
            fn(buf, n, W.SEED, k * n, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            fn(buf, n, W.SEED, (k + 5) * n, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"gsamples_s": n / (ms / 1e3) / 1e9, "gb_s": n * es / (ms / 1e3) / 1e9,
                     "ms_per_launch": ms, "n_per_launch": n, "launch_shape": chosen}
        del buf
    return res


PHILOX_OPS_PER_BLOCK = 40  # 10 rounds x (2 32x32->64 multiplies + 2 three-input XORs)


def alu_peak(z):
    """Lane-level instruction issue peak of the GPU: SMs x 4 schedulers x 32
    lanes x the maximum SM clock (MEASURED_PEAKS.json sm_max_mhz, else the
    device's)."""
    import torch

    props = torch.cuda.get_device_properties(0)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    return props.multi_processor_count * 4 * 32 * mhz * 1e6 / 1e12, mhz


def fused_call(z, dist, dtype, keying, n, seed, offset, sums, hist, ws, stream):
    z.zig_moments_keyed(dist, dtype, keying, n, seed, offset, sums, hist, ws, stream=stream)


def measure_fused(z, stream, reps: int = 5):
    """The fused generate-and-reduce configuration: 2^34 FP32 normals, power
    sums and histogram, nothing stored; per-index and packed keying.  Bound
    by integer issue: the algorithmic work is the Philox blocks (one per
    output per-index, one per 4 outputs packed)."""
    import torch

    c = W.WORKLOADS["normal_f32_fused_2p34"]
    n = c["n"]
    peak, mhz = alu_peak(z)
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    hist = torch.zeros(4098, dtype=torch.int64, device="cuda")
    ws = torch.empty(z.zig_moments_workspace_bytes(c["dist"], c["dtype"]), dtype=torch.uint8,
                     device="cuda")
    res = {}
    for name, keying, blocks in (("per_index", 0, 1.0), ("packed", 1, 0.25)):
        fused_call(z, c["dist"], c["dtype"], keying, n, W.SEED, 0, sums, hist, ws, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(reps):
            fused_call(z, c["dist"], c["dtype"], keying, n, W.SEED, (k + 1) * n, sums, hist, ws,
                       stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        rate = n / (ms / 1e3)
        achieved = rate * blocks * PHILOX_OPS_PER_BLOCK / 1e12
        res[name] = {"gsamples_s": rate / 1e9, "ms_per_launch": ms,
                     "roofline": recorded_pipes("packed" if keying else "index"),
                     "philox_tops": achieved, "lane_issue_peak_tops": peak}
    res["note"] = ("2^34 FP32 normals reduced to 4 power sums and a 4098-bin histogram; "
                   "roofline: the busiest of the integer multiply pipe, the ALU pipe and "
                   "instruction issue in the committed ncu summary of the same kernel source "
                   f"(null if stale); philox_tops counts {PHILOX_OPS_PER_BLOCK} operations per "
                   f"Philox block against SMs x 4 x 32 lanes x {mhz:.0f} MHz")
    return res


def measure_i1024(z, stream, steps: int = 100):
    """The i_max = 1024 tables (zig_generate index_bits 10; different outputs
    from the paper's 256): per-index keying for the four dist/dtype pairs and
    packed keying for FP64, 2^28 counters each, with the HBM-write roofline
    fraction against the measured copy peak."""
    import torch

    peak, _ = measured_peak()
    res = {}
    n = 1 << 28
    for name, dist, dtype, keying in (
            ("exp_f64", W.EXP, W.F64, 0), ("normal_f64", W.NORMAL, W.F64, 0),
            ("exp_f32", W.EXP, W.F32, 0), ("normal_f32", W.NORMAL, W.F32, 0),
            ("exp_f64_packed", W.EXP, W.F64, 1), ("normal_f64_packed", W.NORMAL, W.F64, 1)):
        tdt = torch.float64 if dtype == W.F64 else torch.float32
        es = 8 if dtype == W.F64 else 4
        buf = torch.empty(n, dtype=tdt, device="cuda")

        def call(k):
            z.zig_generate(dist, keying, buf, n, W.SEED, k * n, stream=stream, index_bits=10)

        for k in range(5):
            call(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            call(k + 5)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gbs = n * es / (ms / 1e3) / 1e9
        res[name] = {"gsamples_s": n / (ms / 1e3) / 1e9, "gb_s": gbs, "ms_per_launch": ms,
                     "roofline_frac": gbs / peak}
        del buf
    res["note"] = ("index_bits 10: i_max = 1024 tables (fast path 1020/1024 exponential, "
                   "1021/1024 normal); outputs differ from the 256-slot tables and are checked "
                   "against the oracle on its 10-bit tables")
    return res


def stratified_positions(n: int, m: int, rng_seed: int = 1403):
    """m positions in [0, n), one uniform pick in each of m equal strata."""
    import numpy as np

    rng = np.random.default_rng(rng_seed)
    width = n // m
    return (np.arange(m, dtype=np.uint64) * np.uint64(width)
            + rng.integers(0, width, size=m).astype(np.uint64))


def measure_precision(z, stream, m: int = 1 << 26):
    """The FP32 generator against the FP64 definition of the method, for the
    2^30 counters of each FP32 workload.

    Over the whole range the device's FP32 outputs are compared with its
    FP64 outputs of the same counters (which equal the oracle's: parity
    tests).  On a stratified subset of m counters (one uniform pick in each
    of m equal strata) the oracle itself runs both precisions with its word
    counts: a counter whose FP32 and FP64 draws consume different numbers
    of words took an accept/reject decision the other way (a flip); the
    flipped-decision rate is their share, counted by the oracle.  On the
    same subset the device's FP32 outputs are checked against the oracle's
    FP32 ones and measured in FP32 ulps against its FP64 ones."""
    import numpy as np
    import torch
    from oracle import oracle

    oracle.build()
    res = {}
    chunk = 1 << 26
    for name, dist in (("exp", W.EXP), ("normal", W.NORMAL)):
        c = W.WORKLOADS[f"{name}_f32_2p30"]
        n, off = c["n"], c["offset"]
        fn = z.zig_exponential if dist == W.EXP else z.zig_normal
        x32 = torch.empty(n, dtype=torch.float32, device="cuda")
        x64 = torch.empty(n, dtype=torch.float64, device="cuda")
        fn(x32, n, W.SEED, off, stream=stream)
        fn(x64, n, W.SEED, off, stream=stream)
        torch.cuda.synchronize()
        x0 = float(z.zig_export_tables(dist).X[0])
        max_abs = max_ulp_ge1 = max_ulp_near = 0.0
        same_rn = far = 0
        for k in range(0, n, chunk):
            a = x32[k:k + chunk].double()
            b = x64[k:k + chunk]
            d = (a - b).abs()
            max_abs = max(max_abs, float(d.max()))
            same_rn += int((a == b.float().double()).sum())
            isfar = d > 2.0**-21 * (b.abs() + x0)
            far += int(isfar.sum())
            ulp = torch.ldexp(torch.ones_like(b), torch.frexp(b)[1] - 24)
            r = torch.where(isfar, torch.zeros_like(d), d / ulp)
            max_ulp_near = max(max_ulp_near, float(r.max()))
            big = (b.abs() >= 1.0) & ~isfar
            if bool(big.any()):
                max_ulp_ge1 = max(max_ulp_ge1, float((d / ulp)[big].max()))
        idx = stratified_positions(n, m)
        g32 = x32[torch.from_numpy(idx.astype(np.int64)).cuda()].cpu().numpy()
        del x32, x64
        r32, e32, w32, _ = oracle.fill(dist, W.F32, W.SEED, off, 0, idx=idx, want_words=True)
        r64, e64, w64, _ = oracle.fill(dist, W.F64, W.SEED, off, 0, idx=idx, want_words=True)
        agree = w32 == w64
        flips = int((~agree).sum())
        d = np.abs(g32.astype(np.float64) - r64)
        ulp = np.ldexp(1.0, np.frexp(r64)[1] - 24)
        ratio = np.where(agree, d / ulp, 0.0)
        ge1 = agree & (np.abs(r64) >= 1.0)
        # a zero compares by value: the device's normal zero is +0 whatever
        # the draw's sign (the sign goes inside the one rounding)
        differ = g32.view(np.uint32) != r32.view(np.uint32)
        zero_sign = differ & (g32 == 0) & (r32 == 0)
        res[name] = {
            "n": n, "device_full_range": {
                "max_abs_diff": max_abs, "max_ulp32_where_abs_ge_1": max_ulp_ge1,
                "max_ulp32_agreeing_paths": max_ulp_near,
                "frac_equal_to_rn32_of_fp64": same_rn / n,
                "far_fraction": far / n,
                "far_rule": "|x32 - x64| > 2^-21 (|x64| + X_0): a path change"},
            "oracle_subset": {
                "m": int(idx.size),
                "flipped_decisions": flips, "flipped_decision_rate": flips / idx.size,
                "max_ulp32_vs_fp64_agreeing_paths": float(ratio.max()),
                "max_ulp32_vs_fp64_where_abs_ge_1": float(ratio[ge1].max()) if ge1.any() else 0.0,
                "device_fp32_not_equal_oracle_fp32": int((differ & ~zero_sign).sum()),
                "zeros_differing_in_sign_only": int(zero_sign.sum()),
                "oracle_loop_cap_hits": e32 + e64}}
    torch.cuda.empty_cache()
    res["note"] = (f"flipped_decision_rate: the oracle's FP32 and FP64 word counts differ, on a "
                   f"stratified subset of {m} of the 2^30 counters (one uniform pick per stratum "
                   "of 16); ulp32 = FP32 ulp at the FP64 value. Near zero the FP32 value differs "
                   "from the FP64 one by up to X_i 2^-23 because U keeps its top 23 bits, hence "
                   "large ulp ratios there")
    return res


def measure_packed(z, stream, steps: int = 100):
    """Packed keying (opt-in, different outputs): the four dist/dtype pairs
    at 2^28 counters each through zig_generate, and the FP32 pairs at their
    workload's own launch size, 2^30, with the HBM-write roofline fraction
    of each against the measured copy peak."""
    import torch

    peak, _ = measured_peak()
    res = {}
    for name, dist, dtype, n in (("exp_f64", W.EXP, W.F64, 1 << 28),
                                 ("normal_f64", W.NORMAL, W.F64, 1 << 28),
                                 ("exp_f32", W.EXP, W.F32, 1 << 28),
                                 ("normal_f32", W.NORMAL, W.F32, 1 << 28),
                                 ("exp_f32_2p30", W.EXP, W.F32, 1 << 30),
                                 ("normal_f32_2p30", W.NORMAL, W.F32, 1 << 30)):
        tdt = torch.float64 if dtype == W.F64 else torch.float32
        es = 8 if dtype == W.F64 else 4
        buf = torch.empty(n, dtype=tdt, device="cuda")
        for k in range(5):
            z.zig_generate(dist, z.ZIG_KEY_PACKED, buf, n, W.SEED, k * n, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            z.zig_generate(dist, z.ZIG_KEY_PACKED, buf, n, W.SEED, (k + 5) * n, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        gbs = n * es / (ms / 1e3) / 1e9
        res[name] = {"gsamples_s": n / (ms / 1e3) / 1e9, "gb_s": gbs, "ms_per_launch": ms,
                     "n_per_launch": n, "roofline_frac": gbs / peak}
        del buf
    res["note"] = ("ZIG_KEY_PACKED: one Philox block per 2 FP64 / 4 FP32 fast words; "
                   "outputs differ from per-index keying and are checked against the "
                   "oracle's packed word source")
    return res


def measure_batch(z, stream, reps: int = 10):
    """The batched serving mix (4096 requests, ~3.6e9 variates of mixed
    distribution, precision and parameters) as one zig_batch captured in a
    CUDA graph, against one plain launch per request (also captured), and
    against one large plain launch per (distribution, precision) class
    holding the same number of variates.  Completion times: per request,
    from the batch start (device clock) for zig_batch; from the start event
    for the plain launches (no graph)."""
    import numpy as np
    import torch

    reqs = W.batch_requests()
    total = sum(q["n"] for q in reqs)
    bufs = []
    for q in reqs:
        b = torch.empty(q["n"], dtype=torch.float64 if q["dtype"] else torch.float32, device="cuda")
        q["out"] = b.data_ptr()
        bufs.append(b)
    h = z.pack_requests(reqs)
    d_reqs = torch.from_numpy(h.view(np.uint8)).cuda()
    ws = torch.empty(z.zig_batch_workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    done = torch.zeros(len(reqs), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()

    def timed_graph(fn):
        with torch.cuda.stream(s):
            fn()  # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):  # replays run on the current stream
            g.replay()
            e0.record(s)
            for _ in range(reps):
                g.replay()
            e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def run_batch():
        z.zig_batch(d_reqs, len(reqs), ws, done_ns=done, stream=torch.cuda.current_stream())

    def run_plain():
        cs = torch.cuda.current_stream()
        for q, b in zip(reqs, bufs):
            fn = z.zig_normal if q["dist"] == W.NORMAL else z.zig_exponential
            fn(b, q["n"], q["seed"], q["offset"], stream=cs)

    # the batch's tiles per claim, tuned on this batch before timing
    chunk, chunk_table = z.zig_batch_autotune(d_reqs, len(reqs), ws, reps=3,
                                              stream=torch.cuda.current_stream())
    ms_batch = timed_graph(run_batch)
    lat = done.cpu().numpy().astype(np.float64) / 1e6  # ms from batch start
    ms_plain = timed_graph(run_plain)
    # per-request completion of plain launches (events, no graph)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(reqs) + 1)]
    with torch.cuda.stream(s):
        evs[0].record(s)
        for k, (q, b) in enumerate(zip(reqs, bufs)):
            fn = z.zig_normal if q["dist"] == W.NORMAL else z.zig_exponential
            fn(b, q["n"], q["seed"], q["offset"], stream=s)
            evs[k + 1].record(s)
    torch.cuda.synchronize()
    lat_plain = np.array([evs[0].elapsed_time(e) for e in evs[1:]])
    ms_stream = float(lat_plain[-1])
    # one large plain launch per class with the class's total count
    del bufs
    torch.cuda.empty_cache()
    big_ms = 0.0
    for dist in (W.EXP, W.NORMAL):
        for dtype in (W.F32, W.F64):
            n = sum(q["n"] for q in reqs if q["dist"] == dist and q["dtype"] == dtype)
            b = torch.empty(n, dtype=torch.float64 if dtype else torch.float32, device="cuda")
            fn = z.zig_normal if dist == W.NORMAL else z.zig_exponential
            big_ms += timed_graph(lambda: fn(b, n, 7, 0, stream=torch.cuda.current_stream()))
            del b
    st = z.zig_status_poll()
    rate = total / (ms_batch / 1e3) / 1e9
    return {"requests": len(reqs), "variates": total,
            "bytes": int(sum(q["n"] * (8 if q["dtype"] else 4) for q in reqs)),
            "autotune": {"chosen_chunk_tiles": chunk, "measured": chunk_table},
            "batch_graph": {"ms": ms_batch, "gsamples_s": rate,
                            "p50_ms": float(np.percentile(lat, 50)),
                            "p99_ms": float(np.percentile(lat, 99))},
            "plain_per_request_graph": {"ms": ms_plain,
                                        "gsamples_s": total / (ms_plain / 1e3) / 1e9,
                                        "p50_ms": float(np.percentile(lat_plain, 50)),
                                        "p99_ms": float(np.percentile(lat_plain, 99))},
            "plain_per_request_stream": {"ms": ms_stream,
                                         "gsamples_s": total / (ms_stream / 1e3) / 1e9},
            "plain_large_per_class": {"ms": big_ms, "gsamples_s": total / (big_ms / 1e3) / 1e9},
            "batch_vs_large_plain": (total / (ms_batch / 1e3)) / (total / (big_ms / 1e3)),
            "device_status": z.zig_strerror(st),
            "note": "plain launches produce the standard variates (no scale/location "
                    "transform); the batch applies each request's transform"}


def run_batch_only(args):
    """zig_batch alone on the first K requests of the serving mix: warm-up
    calls, then timed calls with CUDA events (a small case for ncu)."""
    import numpy as np
    import torch

    import paper_1403_6870_gb300 as z

    z.zig_build_tables()
    reqs = W.batch_requests()[:args.batch_requests]
    bufs = []
    for q in reqs:
        b = torch.empty(q["n"], dtype=torch.float64 if q["dtype"] else torch.float32, device="cuda")
        q["out"] = b.data_ptr()
        bufs.append(b)
    d_reqs = torch.from_numpy(z.pack_requests(reqs).view(np.uint8)).cuda()
    ws = torch.empty(z.zig_batch_workspace_bytes(len(reqs)), dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        z.zig_batch(d_reqs, len(reqs), ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        z.zig_batch(d_reqs, len(reqs), ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    total = sum(q["n"] for q in reqs)
    print(json.dumps({"batch_requests": len(reqs), "variates": total, "ms_per_call": ms,
                      "gsamples_s": total / (ms / 1e3) / 1e9,
                      "device_status": z.zig_strerror(z.zig_status_poll())}), flush=True)


def main():
    args = parse_args()
    if args.batch_requests:
        run_batch_only(args)
    elif args.impl == "zig" and "fused" in args.workload:
        run_fused(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_zig(args)


if __name__ == "__main__":
    main()
