#!/usr/bin/env python3
"""Benchmark: GKeys/s of the GB300 sort path on the nine-distribution 1e9-key
int64 workload, with the HBM roofline of its dominant kernel.

One step = one sort of each of the nine seeded 1e9-key int64 arrays (uniform,
Gaussian, sorted, reverse, nearly sorted, 16 distinct, Zipf, all-equal,
uniform [0, 1000)), each read from its own resident input buffer and written
to an output buffer (inputs are 8 GB each, far larger than L2, so no flush is
needed between steps).  Each array is sorted with the parameters of the tuned
table for its sampled distribution class ("tuned", the headline value).  Two
more arms sort the same arrays: "plain", fixed parameters (8-bit digits,
match-mask ranking, default tile: no per-class or per-pass choice), and
"defaults", the library's defaults (adaptive per-pass ranking).  With
--params plain only the fixed-parameter arm runs.

JSON line fields: value (whole-job GKeys/s),
ms_per_step, e2e (same metric through the C ABI with pinned host buffers and
the copies inside the timed region), roofline (dominant kernel, algorithmic
bytes / CUDA-event time vs measured HBM copy bandwidth), cpu_baseline (the CPU
oracle on a bounded sample), clocks, gpu_launches.

    python bench.py                       # N=1, defaults
    python bench.py --impl reference      # the CPU oracle arm
    torchrun --nproc-per-node N bench.py --gpus N   # N replicas, weak scaling
"""
from __future__ import annotations

import argparse
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

DISTS = ["uniform", "gaussian", "sorted", "reverse", "nearly_sorted", "distinct16", "zipf", "equal",
         "uniform1000"]
METRIC = "GKeys/s and % HBM roofline, GA-tuned batched vs plain sort, bit-exact, 1 GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="evosort", choices=["evosort", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000_000, help="keys per array")
    ap.add_argument("--dtype", default="int64", choices=["int32", "int64", "uint32", "uint64"])
    ap.add_argument("--dists", default=",".join(DISTS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-par-sample", type=int, default=1 << 24,
                    help="keys per distribution for the multithreaded CPU baseline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--params", default="auto", choices=["auto", "plain", "tuned"])
    ap.add_argument("--digit-bits", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--kpt", type=int, default=0)
    ap.add_argument("--rank-mode", type=int, default=0)
    ap.add_argument("--pass-kernel", type=int, default=0)
    ap.add_argument("--cpu-sample", type=int, default=1 << 23, help="keys per distribution for the oracle")
    ap.add_argument("--sizes", default="1e7,1e8,1e9,5e9", help="paper9 workload: array sizes")
    ap.add_argument("--workload", default="nine",
                    choices=["nine", "floatpairs", "segmented", "u32big", "paper9", "friendster"],
                    help="nine: the headline workload; the others measure the other configurations")
    ap.add_argument("--segments", type=int, default=100_000)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device) -> float:
    """Max of a per-rank value over all ranks (the step time every rank waits
    for); the identity when no process group is running."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gkeys(keys_per_rank_step: int, world: int, ms_step: float) -> float:
    """Whole-job throughput: keys of all ranks per step over the slowest rank's step time."""
    return keys_per_rank_step * world / (ms_step * 1e-3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def traffic_from_profiles(kernel_src_hash: str):
    """DRAM bytes per key per pass of the onesweep kernel from the committed
    ncu summary, or None if the summary is absent or the kernel has changed."""
    p = os.path.join(ROOT, "profiles", "radix_onesweep_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_sha256") != kernel_src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_key_per_pass"])
    except (KeyError, ValueError):
        return None


def kernel_hash():
    h = hashlib.sha256()
    for f in ("radix.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2505_18681_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Reference arm / CPU baseline: the oracle on a bounded sample of the workload.
# ---------------------------------------------------------------------------
def oracle_sample_run(dists, dtype_name, sample, seed=42):
    import numpy as np
    import torch

    import oracle
    from paper_2505_18681_gb300 import inputs
    tdt = getattr(torch, dtype_name)
    arrays = [inputs.generate(d, sample, tdt, seed=seed, device="cpu").numpy() for d in dists]
    oracle.build()
    t0 = time.perf_counter()
    for a in arrays:
        oracle.radix_sort(a)
    dt = time.perf_counter() - t0
    return len(arrays) * sample, dt


def parallel_sample_run(dists, dtype_name, sample, seed=42):
    """The paper-shaped multithreaded CPU radix sort on every host core, on a
    bounded sample of each distribution: (keys, seconds, threads)."""
    import torch

    import oracle
    from paper_2505_18681_gb300 import inputs
    tdt = getattr(torch, dtype_name)
    arrays = [inputs.generate(d, sample, tdt, seed=seed, device="cpu").numpy() for d in dists]
    oracle.parallel_radix_sort(arrays[0][:1024])   # load, spawn threads once
    used = 1
    t0 = time.perf_counter()
    for a in arrays:
        _, used = oracle.parallel_radix_sort(a)
    dt = time.perf_counter() - t0
    return len(arrays) * sample, dt, used


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    dists = args.dists.split(",")
    sample = args.cpu_sample
    for _ in range(args.warmup):
        oracle_sample_run(dists, args.dtype, sample)
    tot_keys, tot_t = 0, 0.0
    for _ in range(args.steps):
        k, t = oracle_sample_run(dists, args.dtype, sample)
        tot_keys += k
        tot_t += t
    v = tot_keys / tot_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GKeys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic",
        "config": {"workload": "nine-distribution %s sort, oracle on %d keys per distribution per step"
                   % (args.dtype, sample), "n_per_array": sample, "dists": dists},
        "cpu_baseline": {"value": v, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
                         "sample": "%d keys x %d distributions per step, single-threaded C LSD radix"
                         % (sample, len(dists))},
        "e2e": {"value": v, "unit": "GKeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm.
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.workload != "nine":
        other_workload(args)
        return
    import torch
    import torch.distributed as tdist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            tdist.barrier()

    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import inputs
    evo.library()
    dev = torch.device("cuda", local)
    tdt = getattr(torch, args.dtype)
    dists = args.dists.split(",")
    n = args.n
    w = torch.empty(0, dtype=tdt).element_size()

    xs = [inputs.generate(d, n, tdt, seed=42 + 1000 * rank, device=dev) for d in dists]
    out = torch.empty(n, dtype=tdt, device=dev)
    torch.cuda.synchronize()

    kw = {}
    if args.digit_bits:
        kw["digit_bits"] = args.digit_bits
    if args.block:
        kw["block_size"] = args.block
    if args.kpt:
        kw["keys_per_thread"] = args.kpt
    if args.rank_mode:
        kw["rank_mode"] = args.rank_mode
    if args.pass_kernel:
        kw["pass_kernel"] = args.pass_kernel
    stream = torch.cuda.current_stream()
    # plain: one sort call per array with fixed parameters (8-bit digits,
    # match-mask ranking, the default tile), no per-class or per-pass choice
    fixed = {"digit_bits": 8, "rank_mode": 3}
    fixed.update(kw)
    plain = [evo.make_params(algo="radix", stream=stream, **fixed) for _ in dists]
    # the library's defaults (adaptive per-pass ranking), reported beside it
    defaults = [evo.make_params(algo="radix", stream=stream, **kw) for _ in dists]
    params = plain
    mode = "plain"
    table = os.path.join(ROOT, "paper_2505_18681_gb300", "tuned", "gb300_%s.txt" % args.dtype)
    plans = {}
    if args.params in ("auto", "tuned") and not kw and os.path.exists(table):
        # GA-tuned parameters per array, chosen by the dispatcher from each
        # array's sampled distribution class (classified once, before timing)
        evo.table_clear()
        evo.table_load(table)
        params = []
        for d, x in zip(dists, xs):
            pd, cls = evo.plan(x, stream=stream)
            plans[d] = {"class": cls, **pd}
            params.append(evo.make_params(stream=stream, **pd))
        mode = "tuned"
    elif args.params == "tuned":
        raise SystemExit("no tuned table at %s" % table)
    # pre-size the scratch pool so the timed region allocates nothing new
    ws_bytes = max(evo.workspace_bytes(n, tdt, **kw), 1)
    pre = torch.empty(0)
    del pre

    def step(ps):
        for x, p in zip(xs, ps):
            evo.sort(x, out=out, params=p)

    for _ in range(max(args.warmup, 0)):
        step(params)
    evo.sync(stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    launches0 = evo.kernel_launches()
    evo.profile(True)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    # one event per step boundary: the K-step total and each step's time
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for k in range(args.steps):
        step(params)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    e0, e1 = evs[0], evs[-1]
    per_step = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps))
    launches = evo.kernel_launches() - launches0
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync(stream)
    ms = e0.elapsed_time(e1)
    ms_step = max_over_ranks(ms / args.steps, dev)
    keys_per_step = n * len(dists) * ws
    value = whole_job_gkeys(n * len(dists), ws, ms_step)

    # the plain arm (fixed parameters, one sort call per array) and the
    # library-defaults arm on the same inputs, for the tuned-vs-plain comparison
    def time_arm(ps):
        for _ in range(max(args.warmup, 1)):
            step(ps)
        barrier()
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            step(ps)
        p1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(p0.elapsed_time(p1) / args.steps, dev)

    plain_line = defaults_line = None
    if mode == "tuned":
        pms = time_arm(plain)
        plain_line = {"value": keys_per_step / (pms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": pms,
                      "tuned_over_plain": pms / ms_step,
                      "params": "fixed: 8-bit digits, match-mask ranking, default tile"}
        dms = time_arm(defaults)
        defaults_line = {"value": keys_per_step / (dms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": dms,
                         "tuned_over_defaults": dms / ms_step,
                         "params": "library defaults: 8-bit digits, adaptive per-pass ranking, default tile"}

    # dominant kernel: the onesweep pass; time-weighted over active launches
    by_kind = {}
    for r in recs:
        k = by_kind.setdefault(r["kind"], {"ms": 0.0, "bytes": 0.0, "launches": 0, "active": 0})
        k["ms"] += r["ms"]
        k["bytes"] += r["bytes"]
        k["launches"] += 1
        k["active"] += int(r["active"])
    ones = by_kind.get("radix_onesweep", {"ms": 0.0, "bytes": 0.0, "active": 0, "launches": 0})
    act = [r for r in recs if r["kind"] == "radix_onesweep" and r["active"]]
    ach = (sum(r["bytes"] for r in act) / 1e9) / (sum(r["ms"] for r in act) * 1e-3) if act else 0.0
    peak, peak_src = measured_peaks()
    # the committed capture is of the 64-bit keys-only kernel; other key
    # widths have no measured traffic
    tpk = traffic_from_profiles(kernel_hash()) if w == 8 else None
    traffic = None
    if tpk is not None and act:
        traffic = tpk * act[0]["items"]
    total_alg = sum(r["bytes"] for r in recs)
    shares = {k: round(v["ms"] / max(sum(x["ms"] for x in by_kind.values()), 1e-9), 4) for k, v in by_kind.items()}

    # per-distribution device time of one sort each (diagnostic, after the timed region)
    per_dist = {}
    for d, x, p in zip(dists, xs, params):
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        evo.sort(x, out=out, params=p)
        f1.record(stream)
        torch.cuda.synchronize()
        per_dist[d] = round(f0.elapsed_time(f1), 3)

    # end to end: pinned host input -> device, sort, device -> pinned host output
    e2e = None
    if not args.no_e2e and rank == 0 or (not args.no_e2e and ws > 1):
        e2e = measure_e2e(evo, xs, out, params, stream, n, w, args, barrier, ws, dev, mode == "tuned")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        k, t = oracle_sample_run(dists, args.dtype, args.cpu_sample)
        cpu = {"value": k / t / 1e9, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
               "sample": "%d keys of each of the %d distributions (single-threaded C LSD radix, 8-bit digits)"
               % (args.cpu_sample, len(dists))}
        # the paper's multithreaded radix shape on every host core, reported
        # inside the CPU-baseline leg
        k, t, used = parallel_sample_run(dists, args.dtype, args.cpu_par_sample)
        cpu["parallel"] = {"value": k / t / 1e9, "unit": "GKeys/s", "cores": used,
                           "kind": "paper-shaped multithreaded CPU LSD radix (per-thread histograms, "
                                   "thread-wise offsets)",
                           "sample": "%d keys of each of the %d distributions, all online host cores"
                           % (args.cpu_par_sample, len(dists))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GKeys/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "step_ms": {"min": per_step[0], "median": statistics.median(per_step), "max": per_step[-1]},
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "nine-distribution %s sort, %d keys per array (one step sorts all nine)"
                       % (args.dtype, n), "n_per_array": n, "dists": dists, "params": mode,
                       "param_overrides": kw,
                       "tuned_plans": plans,
                       "l2": "inputs larger than L2 (%.1f GB per array), no flush" % (n * w / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "e2e": e2e,
            "plain": plain_line,
            "defaults": defaults_line,
            "roofline": {"bound": "hbm", "kernel": "radix_onesweep", "achieved": ach, "peak": peak,
                         "unit": "GB/s", "frac": ach / peak if peak else None, "traffic": traffic,
                         "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": act[0]["bytes"] if act else None,
                         "avg_active_launch_ms": (sum(r["ms"] for r in act) / len(act)) if act else None},
            "whole_step_alg_gbs": total_alg / args.steps / 1e9 / (ms_step * 1e-3),
            "kernel_time_share": shares,
            "per_dist_ms": per_dist,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.destroy_process_group()


def measure_e2e(evo, xs, out, params, stream, n, w, args, barrier, ws, dev, auto):
    """The same step through the C-ABI host-memory entry point: each array's
    keys go from page-locked host memory to the device, are sorted there and
    come back to host memory, with the copies of neighbouring arrays
    overlapping the sorts (evosort_sort_host_batch)."""
    import torch
    try:
        host_in = [x.cpu().pin_memory() for x in xs]
    except RuntimeError:
        return None
    host_out = torch.empty(n, dtype=xs[0].dtype).pin_memory()
    # tuned: AUTO parameters, so the library plans each array from a host sample
    p = evo.make_params(stream=stream) if auto else params[0]

    def step():
        evo.sort_host_batch(host_in, [host_out] * len(host_in), params=p)

    step()
    evo.sync(stream)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 3))
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    evo.sync(stream)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    keys = n * len(xs) * ws
    del host_in, host_out
    return {"value": keys / (ms * 1e-3) / 1e9, "unit": "GKeys/s", "h2d_bytes_per_step": n * w * len(xs),
            "d2h_bytes_per_step": n * w * len(xs), "ms_per_step": ms, "steps": steps,
            "path": "evosort_sort_host_batch: page-locked host arrays in and out, uploads and downloads "
                    "overlapping the sorts"}


# ---------------------------------------------------------------------------
# The other configurations (one JSON line each; not the headline bench line).
# ---------------------------------------------------------------------------
def _time_steps(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def other_workload(args):
    import torch

    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import inputs
    evo.library()
    stream = torch.cuda.current_stream()
    peak, peak_src = measured_peaks()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    line = {"metric": METRIC, "unit": "GKeys/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    if args.workload == "floatpairs":
        n = 500_000_000 if args.n == 1_000_000_000 else args.n
        x = inputs.generate("float_mix", n, torch.float64, seed=42, device="cuda")
        v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
        ko, vo = torch.empty_like(x), torch.empty_like(v)
        p = evo.make_params(algo="radix", stream=stream)
        launches0 = evo.kernel_launches()
        evo.profile(True)
        sampler.start()
        ms = _time_steps(lambda: evo.sort_pairs(x, v, ko, vo, params=p), args.steps, args.warmup, stream)
        clocks = sampler.stop()
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep" and r["active"]]
        evo.profile(False)
        evo.sync()
        ach = sum(r["bytes"] for r in recs) / 1e9 / (sum(r["ms"] for r in recs) * 1e-3) if recs else 0.0
        line.update(value=n / (ms * 1e-3) / 1e9, ms_per_step=ms, dtype="f64+u32",
                    config={"workload": "stable key/value argsort, %d float64 keys (uniform [-1e6,1e6], 1%% "
                            "duplicates, -0.0/+0.0/NaN sprinkled) with uint32 index payload" % n},
                    roofline={"bound": "hbm", "kernel": "radix_onesweep (pairs)", "achieved": ach, "peak": peak,
                              "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": peak_src},
                    clocks=clocks, gpu_launches=evo.kernel_launches() - launches0)
    elif args.workload == "paper9":
        # the paper's nine int32 distributions over a size sweep, five timed
        # sorts each (the paper's protocol: min / median / max of 5), tuned
        # int32 table through the dispatcher
        sizes = [int(float(v)) for v in args.sizes.split(",")]
        table = os.path.join(ROOT, "paper_2505_18681_gb300", "tuned", "gb300_int32.txt")
        evo.table_clear()
        if os.path.exists(table):
            evo.table_load(table)
        res = {}
        tot_keys = tot_ms = 0.0
        launches0 = evo.kernel_launches()
        sampler.start()
        for d in inputs.PAPER_DISTRIBUTIONS:
            res[d] = {}
            for n in sizes:
                x = inputs.generate(d, n, torch.int32, seed=42, device="cuda")
                y = torch.empty_like(x)
                pd, _ = evo.plan(x, stream=stream)
                p = evo.make_params(stream=stream, **pd)
                for _ in range(max(args.warmup, 1)):
                    evo.sort(x, out=y, params=p)
                ts = []
                for _ in range(5):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    evo.sort(x, out=y, params=p)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
                evo.sync()
                ts.sort()
                res[d]["%.0e" % n] = {"min_ms": round(ts[0], 4), "median_ms": round(ts[2], 4),
                                      "max_ms": round(ts[4], 4)}
                tot_keys += n
                tot_ms += ts[2]
                del x, y
                torch.cuda.empty_cache()
        clocks = sampler.stop()
        evo.table_clear()
        line.update(value=tot_keys / (tot_ms * 1e-3) / 1e9, ms_per_step=tot_ms, dtype="i32",
                    config={"workload": "the paper's nine int32 distributions in [-1e9, 1e9], sizes %s, "
                            "median of 5 sorts each, tuned int32 table" % args.sizes},
                    per_dist=res, clocks=clocks, gpu_launches=evo.kernel_launches() - launches0)
    elif args.workload == "friendster":
        # stand-in for the paper's real-data test: 3,612,134,270 int32 node
        # ids of a heavy-tailed graph, one sort, tuned int32 table
        n = inputs.FRIENDSTER_N if args.n == 1_000_000_000 else args.n
        table = os.path.join(ROOT, "paper_2505_18681_gb300", "tuned", "gb300_int32.txt")
        evo.table_clear()
        if os.path.exists(table):
            evo.table_load(table)
        x = inputs.generate("friendster_like", n, torch.int32, seed=42, device="cuda")
        y = torch.empty_like(x)
        pd, cls = evo.plan(x, stream=stream)
        p = evo.make_params(stream=stream, **pd)
        launches0 = evo.kernel_launches()
        evo.profile(True)
        sampler.start()
        ms = _time_steps(lambda: evo.sort(x, out=y, params=p), args.steps, args.warmup, stream)
        clocks = sampler.stop()
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep" and r["active"]]
        evo.profile(False)
        evo.sync()
        evo.table_clear()
        ach = sum(r["bytes"] for r in recs) / 1e9 / (sum(r["ms"] for r in recs) * 1e-3) if recs else 0.0
        line.update(value=n / (ms * 1e-3) / 1e9, ms_per_step=ms, dtype="i32",
                    config={"workload": "%d int32 node ids in [101, 124836179] with heavy-tailed frequency "
                            "(stand-in for the paper's Friendster endpoint column), one sort" % n,
                            "class": cls, "plan": pd},
                    roofline={"bound": "hbm", "kernel": "radix_onesweep", "achieved": ach, "peak": peak,
                              "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": peak_src},
                    clocks=clocks, gpu_launches=evo.kernel_launches() - launches0)
    elif args.workload == "u32big":
        n = 10_000_000_000 if args.n == 1_000_000_000 else args.n
        x = inputs.generate("uniform", n, torch.uint32, seed=42, device="cuda")
        y = torch.empty_like(x)
        p = evo.make_params(algo="radix", stream=stream)
        launches0 = evo.kernel_launches()
        evo.profile(True)
        sampler.start()
        ms = _time_steps(lambda: evo.sort(x, out=y, params=p), args.steps, args.warmup, stream)
        clocks = sampler.stop()
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep" and r["active"]]
        evo.profile(False)
        evo.sync()
        ach = sum(r["bytes"] for r in recs) / 1e9 / (sum(r["ms"] for r in recs) * 1e-3) if recs else 0.0
        line.update(value=n / (ms * 1e-3) / 1e9, ms_per_step=ms, dtype="u32",
                    config={"workload": "%d uint32 keys uniform (%.0f GB, double-buffered in HBM), one sort"
                            % (n, n * 4 / 1e9)},
                    roofline={"bound": "hbm", "kernel": "radix_onesweep", "achieved": ach, "peak": peak,
                              "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": peak_src},
                    clocks=clocks, gpu_launches=evo.kernel_launches() - launches0)
    else:   # segmented
        lens = inputs.segment_lengths(args.segments, 16, 1_000_000, seed=42)
        keys, offs = inputs.segmented_keys(lens, torch.int32, seed=42, device="cuda")
        d_offs = offs.to("cuda")
        total = keys.numel()
        work = torch.empty_like(keys)
        # tier threshold chosen by timing every allowed value (the batched path's only knob)
        best_cap, best_ms = None, None
        for cap in (1024, 2048, 4096, 8192):
            p = evo.make_params(seg_block_cap=cap, stream=stream)

            def run_batched(p=p):
                work.copy_(keys)
                evo.segmented_sort(work, d_offs, params=p)
            t = _time_steps(run_batched, 1, 1, stream)
            if best_ms is None or t < best_ms:
                best_cap, best_ms = cap, t
        p = evo.make_params(seg_block_cap=best_cap, stream=stream)
        copy_ms = _time_steps(lambda: work.copy_(keys), args.steps, 1, stream)

        def run_batched():
            work.copy_(keys)
            evo.segmented_sort(work, d_offs, params=p)
        launches0 = evo.kernel_launches()
        sampler.start()
        ms = _time_steps(run_batched, args.steps, args.warmup, stream) - copy_ms
        clocks = sampler.stop()
        batched_launches = (evo.kernel_launches() - launches0) // (args.steps + args.warmup)
        # plain path: one default sort call per array
        bounds = offs.tolist()
        plain_p = evo.make_params(algo="radix", stream=stream)

        def run_plain():
            work.copy_(keys)
            for i in range(len(bounds) - 1):
                a, b = bounds[i], bounds[i + 1]
                if b - a > 1:
                    evo.sort(work[a:b], params=plain_p)
        plain_ms = _time_steps(run_plain, 1, 1, stream) - copy_ms
        evo.sync()
        line.update(value=total / (ms * 1e-3) / 1e9, ms_per_step=ms, dtype="i32",
                    config={"workload": "batched segmented sort: %d int32 arrays, log-uniform lengths 16..1e6, "
                            "%d keys total, even arrays uniform, odd nearly sorted" % (args.segments, total),
                            "seg_block_cap": best_cap, "launches_per_batched_sort": batched_launches},
                    plain={"value": total / (plain_ms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": plain_ms,
                           "batched_over_plain": plain_ms / ms, "calls": len(bounds) - 1},
                    clocks=clocks)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
