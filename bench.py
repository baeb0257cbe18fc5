#!/usr/bin/env python3
"""Benchmark: GKeys/s of the GB300 sort path on the nine-distribution 1e9-key
int64 workload, with the HBM roofline of its dominant kernel, and the other
configurations measured beside it.

Headline step (value): one sort of each of the nine seeded 1e9-key int64
arrays (uniform, Gaussian, sorted, reverse, nearly sorted, 16 distinct, Zipf,
all-equal, uniform [0, 1000)), each read from its own resident input buffer
and written to an output buffer (inputs are 8 GB each, far larger than L2, so
no flush is needed between steps).  Each sort is the call a user makes with
the choice left to the library: the dispatcher samples the array, classifies
it and takes the GA-tuned table's parameters ("tuned").  Two more arms sort
the same arrays: "plain", fixed parameters (8-bit digits, match-mask ranking,
the default tile: no per-class or per-pass choice), and "defaults", the
library's built-in parameters.

The other configurations run after the headline (single GPU only) and are
reported as sub-objects of the same JSON line: "int32" (the same nine
distributions as 1e9-key int32 arrays, with its own roofline), "floatpairs"
(5e8 float64 keys with a uint32 index, stable), "segmented" (100,000 int32
arrays of log-uniform length 16..1e6, one batched call, tuned vs defaults vs
one call per array), "u32big" (1e10 uint32 keys in one sort), "small" (latency
of 1e3..1e4-key sorts through the one-CTA path against the radix path) and
"merge" (mergesort of 1e8 int32 keys).

JSON line fields: value (whole-job GKeys/s), ms_per_step, e2e (same metric
through the C ABI with pinned host buffers and the copies inside the timed
region), roofline (dominant kernel, algorithmic bytes / CUDA-event time vs
measured HBM copy bandwidth), cpu_baseline (the CPU oracle on a bounded
sample), clocks, gpu_launches, and the sub-objects above.

    python bench.py                       # N=1, defaults
    python bench.py --no-extras           # the headline only
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
    ap.add_argument("--no-extras", action="store_true", help="measure the headline configuration only")
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
                    choices=["nine", "int32", "floatpairs", "segmented", "u32big", "small", "merge", "serving",
                             "paper9", "friendster"],
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


def kernel_hash():
    h = hashlib.sha256()
    for f in ("onesweep_reg.cuh", "radix.cuh", "common.cuh"):
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
TABLE_DIR = os.path.join(ROOT, "paper_2505_18681_gb300", "tuned")


def traffic_per_key_pass(w: int):
    """DRAM bytes per key per pass of the register-tile onesweep kernel for
    key width w, from the committed ncu summary of that width, or None if the
    summary is absent or the kernel source has changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "radix_onesweep_reg_int%d.txt" % (8 * w))
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_sha256") != kernel_hash():
        return None
    try:
        return float(vals["dram_bytes_per_key_per_pass"])
    except (KeyError, ValueError):
        return None


def onesweep_roofline(recs, w, peak, peak_src):
    """Roofline of the dominant kernel (the onesweep pass) over the active
    launches of a timed region: algorithmic bytes / CUDA-event time."""
    act = [r for r in recs if r["kind"] == "radix_onesweep" and r["active"]]
    ach = (sum(r["bytes"] for r in act) / 1e9) / (sum(r["ms"] for r in act) * 1e-3) if act else 0.0
    tpk = traffic_per_key_pass(w)
    traffic = tpk * act[0]["items"] if (tpk is not None and act) else None
    return {"bound": "hbm", "kernel": "radix_onesweep", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if peak else None, "traffic": traffic, "peak_source": peak_src,
            "algorithmic_bytes_per_launch": act[0]["bytes"] if act else None,
            "avg_active_launch_ms": (sum(r["ms"] for r in act) / len(act)) if act else None,
            "active_launches": len(act)}


def kernel_shares(recs):
    by_kind = {}
    for r in recs:
        by_kind[r["kind"]] = by_kind.get(r["kind"], 0.0) + r["ms"]
    tot = max(sum(by_kind.values()), 1e-9)
    return {k: round(v / tot, 4) for k, v in by_kind.items()}


def time_region(fn, steps, stream):
    """Device time of `steps` calls of fn between two events on `stream`, and
    the per-step times (one event per step boundary)."""
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for k in range(steps):
        fn()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    per = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(steps))
    return evs[0].elapsed_time(evs[-1]), per


def nine_leg(evo, args, dtype_name, n, dists, stream, rank, ws, barrier, dev, keep_inputs=False):
    """The nine-distribution step for one key type: tuned (dispatcher call),
    plain and defaults arms, per-distribution times, roofline of the dominant
    kernel, kernel shares and clocks.  Returns (fields, inputs or None)."""
    import torch
    from paper_2505_18681_gb300 import inputs
    tdt = getattr(torch, dtype_name)
    w = torch.empty(0, dtype=tdt).element_size()
    xs = [inputs.generate(d, n, tdt, seed=42 + 1000 * rank, device=dev) for d in dists]
    out = torch.empty(n, dtype=tdt, device=dev)
    torch.cuda.synchronize()
    kw = {}
    for k, a in (("digit_bits", args.digit_bits), ("block_size", args.block), ("keys_per_thread", args.kpt),
                 ("rank_mode", args.rank_mode), ("pass_kernel", args.pass_kernel)):
        if a:
            kw[k] = a
    # plain: one sort call per array with fixed parameters (8-bit digits,
    # match-mask ranking, the default tile), no per-class or per-pass choice
    fixed = {"digit_bits": 8, "rank_mode": 3}
    fixed.update(kw)
    plain = evo.make_params(algo="radix", stream=stream, **fixed)
    defaults = evo.make_params(algo="radix", stream=stream, **kw)
    table = os.path.join(TABLE_DIR, "gb300_%s.txt" % dtype_name)
    evo.table_clear()
    mode = "plain"
    tuned = plain
    plans = {}
    if args.params in ("auto", "tuned") and not kw and os.path.exists(table):
        # the call a user makes: AUTO parameters, so the dispatcher samples
        # each array, classifies it and takes the tuned table's entry
        evo.table_load(table)
        tuned = evo.make_params(stream=stream)
        mode = "tuned"
        for d, x in zip(dists, xs):
            pd, cls = evo.plan(x, stream=stream)
            plans[d] = {"class": cls, **pd}
    elif args.params == "tuned":
        raise SystemExit("no tuned table at %s" % table)

    def step(p):
        for x in xs:
            evo.sort(x, out=out, params=p)

    for _ in range(max(args.warmup, 0)):
        step(tuned)
    evo.sync(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    launches0 = evo.kernel_launches()
    evo.profile(True)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ms, per_step = time_region(lambda: step(tuned), args.steps, stream)
    barrier()
    clocks = sampler.stop()
    launches = evo.kernel_launches() - launches0
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync(stream)
    ms_step = max_over_ranks(ms / args.steps, dev)
    keys_per_step = n * len(dists) * ws

    def time_arm(p):
        for _ in range(max(args.warmup, 1)):
            step(p)
        barrier()
        torch.cuda.synchronize()
        t, _ = time_region(lambda: step(p), args.steps, stream)
        return max_over_ranks(t / args.steps, dev)

    plain_line = defaults_line = None
    if mode == "tuned":
        pms = time_arm(plain)
        plain_line = {"value": keys_per_step / (pms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": pms,
                      "tuned_over_plain": pms / ms_step,
                      "params": "fixed: 8-bit digits, match-mask ranking, default tile"}
        dms = time_arm(defaults)
        defaults_line = {"value": keys_per_step / (dms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": dms,
                         "tuned_over_defaults": dms / ms_step,
                         "params": "library defaults: 8-bit digits, register tile, adaptive per-pass ranking"}
    peak, peak_src = measured_peaks()
    per_dist = {}
    for d, x in zip(dists, xs):
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        evo.sort(x, out=out, params=tuned)
        f1.record(stream)
        torch.cuda.synchronize()
        per_dist[d] = round(f0.elapsed_time(f1), 3)
    fields = {
        "value": whole_job_gkeys(n * len(dists), ws, ms_step), "ms_per_step": ms_step,
        "step_ms": {"min": per_step[0], "median": statistics.median(per_step), "max": per_step[-1]},
        "config": {"workload": "nine-distribution %s sort, %d keys per array (one step sorts all nine)"
                   % (dtype_name, n), "n_per_array": n, "dists": dists, "params": mode,
                   "param_overrides": kw, "tuned_plans": plans,
                   "l2": "inputs larger than L2 (%.1f GB per array), no flush" % (n * w / 1e9)},
        "plain": plain_line, "defaults": defaults_line,
        "roofline": onesweep_roofline(recs, w, peak, peak_src),
        "whole_step_alg_gbs": sum(r["bytes"] for r in recs) / args.steps / 1e9 / (ms_step * 1e-3),
        "kernel_time_share": kernel_shares(recs), "per_dist_ms": per_dist, "clocks": clocks,
        "gpu_launches": launches, "_tuned_params": tuned,
    }
    if keep_inputs:
        return fields, (xs, out)
    del xs, out
    return fields, None


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
    evo.library()
    dev = torch.device("cuda", local)
    dists = args.dists.split(",")
    stream = torch.cuda.current_stream()
    head, kept = nine_leg(evo, args, args.dtype, args.n, dists, stream, rank, ws, barrier, dev, keep_inputs=True)
    xs, out = kept
    w = xs[0].element_size()

    # end to end: pinned host input -> device, sort, device -> pinned host output
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(evo, xs, out, [head["_tuned_params"]] * len(xs), stream, args.n, w, args, barrier, ws,
                          dev, head["config"]["params"] == "tuned")
    del xs, out, kept
    torch.cuda.empty_cache()

    extras = {}
    if ws == 1 and not args.no_extras:
        for name, fn in (("int32", leg_int32), ("floatpairs", leg_floatpairs), ("segmented", leg_segmented),
                         ("u32big", leg_u32big), ("small", leg_small), ("merge", leg_merge),
                         ("serving", leg_serving)):
            try:
                extras[name] = fn(evo, args, stream, barrier, dev)
            except Exception as exc:   # one configuration's failure does not drop the line
                extras[name] = {"error": "%s: %s" % (type(exc).__name__, str(exc)[:300])}
            torch.cuda.empty_cache()
        evo.table_clear()

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
        cfg = head["config"]
        cfg["parallelism"] = "replicas" if ws > 1 else "single GPU"
        line = {
            "metric": METRIC, "value": head["value"], "unit": "GKeys/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "step_ms": head["step_ms"], "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic", "config": cfg, "e2e": e2e, "plain": head["plain"], "defaults": head["defaults"],
            "roofline": head["roofline"], "whole_step_alg_gbs": head["whole_step_alg_gbs"],
            "kernel_time_share": head["kernel_time_share"], "per_dist_ms": head["per_dist_ms"],
            "cpu_baseline": cpu, "clocks": head["clocks"], "gpu_launches": head["gpu_launches"],
        }
        line.update(extras)
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
# The other configurations, measured after the headline on one GPU.
# ---------------------------------------------------------------------------
def leg_int32(evo, args, stream, barrier, dev):
    """The nine distributions as 1e9-key int32 arrays (the configuration the
    60%-of-HBM target is set on), with its own roofline."""
    fields, _ = nine_leg(evo, args, "int32", args.n, args.dists.split(","), stream, 0, 1, barrier, dev)
    fields.pop("_tuned_params", None)
    return fields


def _timed_with_profile(evo, fn, steps, warmup, stream):
    import torch
    for _ in range(max(warmup, 1)):
        fn()
    evo.sync(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    launches0 = evo.kernel_launches()
    evo.profile(True)
    sampler.start()
    ms, _ = time_region(fn, steps, stream)
    clocks = sampler.stop()
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync(stream)
    return ms / steps, recs, clocks, evo.kernel_launches() - launches0


def leg_floatpairs(evo, args, stream, barrier, dev):
    """5e8 float64 keys (uniform [-1e6, 1e6], 1% duplicates, -0.0/+0.0/NaN
    sprinkled) with a uint32 index payload: the stable argsort."""
    import torch
    from paper_2505_18681_gb300 import inputs
    n = 500_000_000
    x = inputs.generate("float_mix", n, torch.float64, seed=42, device=dev)
    v = torch.arange(n, dtype=torch.int64, device=dev).to(torch.int32).view(torch.uint32)
    ko, vo = torch.empty_like(x), torch.empty_like(v)
    p = evo.make_params(stream=stream)
    ms, recs, clocks, launches = _timed_with_profile(evo, lambda: evo.sort_pairs(x, v, ko, vo, params=p),
                                                     args.steps, args.warmup, stream)
    peak, src = measured_peaks()
    roof = onesweep_roofline(recs, 8, peak, src)
    roof["kernel"] = "radix_onesweep (key/value)"
    roof["traffic"] = None
    return {"value": n / (ms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms, "dtype": "f64+u32",
            "config": {"workload": "stable key/value argsort, %d float64 keys with uint32 index payload" % n},
            "roofline": roof, "kernel_time_share": kernel_shares(recs), "clocks": clocks,
            "gpu_launches": launches}


def segmented_block_cap(path, w, total):
    """seg_block_cap of the tuned segmented entry (class 8) nearest to the
    batch's size bucket in a table file (the library default if none)."""
    dt_code = 0 if w == 4 else 1
    best = None
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            v = line.split()
            if int(v[0]) == dt_code and int(v[2]) == 8:
                d = abs(int(v[1]) - (max(total, 1).bit_length() - 1))
                if best is None or d < best[0]:
                    best = (d, int(v[9]))
    return best[1] if best and best[1] > 0 else (8192 if w == 4 else 4096)


def segmented_alg_bytes(lens, w, block_cap):
    """Algorithmic bytes of one batched segmented sort: 2w per key for a
    segment one CTA sorts on chip, and the radix formula w + P * 2w per key
    (P = 8w / 8 passes of 8-bit digits, all active for full-range keys) for
    the longer ones."""
    import torch
    lens = torch.as_tensor(lens, dtype=torch.int64)
    small = int(lens[lens <= block_cap].sum())
    big = int(lens[lens > block_cap].sum())
    return 2 * w * small + (w + w * 2 * w) * big


def leg_segmented(evo, args, stream, barrier, dev, nseg=100_000, rank=0, world=1):
    """100,000 int32 arrays with log-uniform lengths 16..1e6 (half uniform,
    half nearly sorted): one batched call with the GA-tuned cut-overs against
    the built-in ones and against one sort call per array.  With world > 1
    ranks the batch is sharded by whole segments (longest first, to the rank
    with the fewest keys): each rank generates and sorts only its own share,
    nothing is exchanged, and the value is all keys over the slowest rank's
    time (strong scaling)."""
    import torch
    from paper_2505_18681_gb300 import inputs, shard
    lens = inputs.segment_lengths(nseg, 16, 1_000_000, seed=42)
    loads = None
    if world > 1:
        owned, loads = shard.partition_segments(lens, world)
        keys, offs = shard.rank_batch(lens, owned[rank], torch.int32, seed=42, device=dev)
    else:
        keys, offs = inputs.segmented_keys(lens, torch.int32, seed=42, device=dev)
    d_offs = offs.to(dev)
    total_all = int(lens.sum())
    total = keys.numel()
    work = torch.empty_like(keys)
    evo.table_clear()
    evo.table_load(os.path.join(TABLE_DIR, "gb300_int32.txt"))
    tuned = evo.make_params(stream=stream)                 # AUTO: the table's segmented entry
    defaults = evo.make_params(algo="radix", stream=stream)
    copy_ms = _time_steps(lambda: work.copy_(keys), args.steps, 1, stream)

    def batched(p):
        def f():
            work.copy_(keys)
            evo.segmented_sort(work, d_offs, params=p)
        return f
    barrier()
    ms_t, recs, clocks, launches = _timed_with_profile(evo, batched(tuned), args.steps, args.warmup, stream)
    barrier()
    ms_t = max_over_ranks(ms_t - copy_ms, dev)
    if world > 1:
        evo.table_clear()
        return {"value": total_all / (ms_t * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms_t, "dtype": "i32",
                "n_gpus": world, "scaling": "strong",
                "config": {"workload": "batched segmented sort: %d int32 arrays, log-uniform lengths 16..1e6, %d "
                           "keys total, sharded over %d ranks by whole segments (no exchange)"
                           % (nseg, total_all, world), "keys_per_rank": loads},
                "kernel_time_share": kernel_shares(recs), "clocks": clocks}
    ms_d = _time_steps(batched(defaults), args.steps, 1, stream) - copy_ms
    # the tuned batch captured once into a CUDA graph and replayed (the call
    # captures: its scratch comes from the stream-ordered pool and it reads
    # nothing back); the replay includes the input copy, subtracted as above
    gs = torch.cuda.Stream()
    gs.wait_stream(stream)
    gp = evo.make_params(stream=gs)
    with torch.cuda.stream(gs):
        evo.segmented_sort(work, d_offs, params=gp)   # pool warm-up outside the capture
        gs.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            work.copy_(keys)
            evo.segmented_sort(work, d_offs, params=gp)
    stream.wait_stream(gs)
    ms_g = _time_steps(graph.replay, args.steps, 1, stream) - copy_ms
    evo.sync()
    del graph
    # one sort call per array with the library's own choice (no table: the
    # one-CTA path for short arrays, the device-wide radix sort for the rest)
    evo.table_clear()
    bounds = offs.tolist()
    plain_p = evo.make_params(stream=stream)

    def per_array():
        work.copy_(keys)
        for i in range(len(bounds) - 1):
            a, b = bounds[i], bounds[i + 1]
            if b - a > 1:
                evo.sort(work[a:b], params=plain_p)
    plain_ms = _time_steps(per_array, 1, 1, stream) - copy_ms
    evo.sync()
    cap = segmented_block_cap(os.path.join(TABLE_DIR, "gb300_int32.txt"), 4, total)
    alg = segmented_alg_bytes(lens, 4, cap)
    peak, peak_src = measured_peaks()
    ach = alg / 1e9 / (ms_t * 1e-3)
    seg_roof = {"bound": "hbm", "kernel": "seg_sort (whole batch, one persistent launch)", "achieved": ach,
                "peak": peak, "unit": "GB/s", "frac": ach / peak if peak else None, "traffic": None,
                "peak_source": peak_src, "algorithmic_bytes_per_batch": alg, "block_cap": cap}
    return {"value": total / (ms_t * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms_t, "dtype": "i32",
            "config": {"workload": "batched segmented sort: %d int32 arrays, log-uniform lengths 16..1e6, %d keys "
                       "total, even arrays uniform, odd nearly sorted" % (nseg, total),
                       "tuned_params": "GA table entry for segmented batches (class 'segmented')"},
            "defaults": {"value": total / (ms_d * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms_d,
                         "tuned_over_defaults": ms_d / ms_t},
            "graph": {"value": total / (ms_g * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms_g,
                      "path": "the tuned batch captured once into a CUDA graph, replayed each step"},
            "roofline": seg_roof,
            "plain": {"value": total / (plain_ms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": plain_ms,
                      "batched_over_plain": plain_ms / ms_t, "calls": len(bounds) - 1,
                      "params": "one sort call per array, library defaults"},
            "kernel_time_share": kernel_shares(recs), "clocks": clocks, "gpu_launches_per_batch": launches /
            max(args.steps, 1)}


def leg_u32big(evo, args, stream, barrier, dev):
    """1e10 uint32 keys uniform (40 GB, double-buffered in HBM), one sort."""
    import torch
    from paper_2505_18681_gb300 import inputs
    n = 10_000_000_000
    x = inputs.generate("uniform", n, torch.uint32, seed=42, device=dev)
    y = torch.empty_like(x)
    p = evo.make_params(stream=stream)
    ms, recs, clocks, launches = _timed_with_profile(evo, lambda: evo.sort(x, out=y, params=p),
                                                     max(1, min(args.steps, 3)), 1, stream)
    peak, src = measured_peaks()
    roof = onesweep_roofline(recs, 4, peak, src)
    roof["traffic"] = None   # 64-bit look-back slots at this size: not the captured kernel configuration
    return {"value": n / (ms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms, "dtype": "u32",
            "config": {"workload": "%d uint32 keys uniform (%.0f GB, double-buffered in HBM), one sort"
                       % (n, n * 4 / 1e9)},
            "roofline": roof, "kernel_time_share": kernel_shares(recs), "clocks": clocks,
            "gpu_launches": launches}


def small_graph_us(evo, x, y, kw, reps=100):
    """Device time of one sort with no host in the loop: `reps` sorts captured
    in one CUDA graph on a side stream, the graph replayed and timed with
    events (median of 5 replays), divided by reps."""
    import torch
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    q = evo.make_params(stream=gs, **kw)
    with torch.cuda.stream(gs):
        evo.sort(x, out=y, params=q)          # pool warm-up outside the capture
        gs.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            for _ in range(reps):
                evo.sort(x, out=y, params=q)
        g.replay()
        gs.synchronize()
        ts = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(gs)
            g.replay()
            e1.record(gs)
            gs.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3 / reps)
    torch.cuda.current_stream().wait_stream(gs)
    del g
    return statistics.median(ts)


def leg_small(evo, args, stream, barrier, dev):
    """Latency of small sorts: the dispatcher's one-CTA path (the default for
    arrays up to 4096 keys) against the device-wide radix path, per call."""
    import torch
    from paper_2505_18681_gb300 import inputs
    # no tuned table: above the one-CTA cut-over 'auto' then takes the default
    # radix plan with no sample of the keys (a sample reads back to the host,
    # which a graph capture does not allow)
    evo.table_clear()
    res = {}
    for n in (1000, 4096, 10_000):
        x = inputs.generate("uniform", n, torch.int32, seed=42, device=dev)
        y = torch.empty_like(x)
        row = {}
        for label, kw in (("auto", {}), ("radix", {"algo": "radix"})):
            p = evo.make_params(stream=stream, **kw)
            for _ in range(20):
                evo.sort(x, out=y, params=p)
            torch.cuda.synchronize()
            dev_us, host_us = [], []
            k0 = evo.kernel_launches()
            evo.profile(True)
            for _ in range(101):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                e0.record(stream)
                evo.sort(x, out=y, params=p)
                e1.record(stream)
                torch.cuda.synchronize()
                host_us.append((time.perf_counter() - t0) * 1e6)
                dev_us.append(e0.elapsed_time(e1) * 1e3)
            recs = evo.profile_read()
            evo.profile(False)
            row[label] = {"call_us_median": statistics.median(dev_us), "host_us_median": statistics.median(host_us),
                          "kernel_us_per_call": sum(r["ms"] for r in recs) * 1e3 / 101,
                          "launches_per_call": (evo.kernel_launches() - k0) / 101,
                          "graph_us_per_sort": small_graph_us(evo, x, y, kw)}
        res[str(n)] = row
    return {"unit": "us per sort", "config": {"workload": "one int32 array of 1e3 / 4096 / 1e4 uniform keys per call; "
                                              "'auto' lets the dispatcher choose (one-CTA path up to 4096 keys), "
                                              "'radix' forces the device-wide radix sort; call_us: events around "
                                              "the Python call on its stream (includes host overhead), "
                                              "kernel_us: the library's events around its launches (includes "
                                              "launch latency), graph_us: device time per sort from a replayed "
                                              "CUDA graph of 100 sorts"},
            "latency": res}


def leg_serving(evo, args, stream, barrier, dev, requests=300):
    """The serving loop on a Poisson stream of sort requests, sizes
    log-uniform 1e3..1e8 keys, dtypes int32 / int64 / float64, at 70% of the
    measured capacity: p50/p99 latency (arrival to completion) and keys/s."""
    from paper_2505_18681_gb300 import serve
    evo.table_clear()
    evo.table_load(os.path.join(TABLE_DIR, "gb300_int32.txt"))   # tuned entries of both key widths
    res = serve.serve_mix(requests, 100_000_000, table=os.path.join(TABLE_DIR, "gb300_int64.txt"))
    evo.table_clear()
    return {"value": res["keys_per_s"] / 1e9, "unit": "GKeys/s", "p50_ms": res["p50_ms"], "p99_ms": res["p99_ms"],
            "config": {"workload": "%d sort requests, log-uniform sizes 1e3..1e8 keys (largest %d), int32 / int64 / "
                       "float64, Poisson arrivals at %.0f%% of the measured capacity" % (
                           requests, res["largest_request"], 100 * res["load"])},
            "detail": res}


def leg_merge(evo, args, stream, barrier, dev):
    """Mergesort (Algorithm 3) of 1e8 int32 keys, insertion threshold 32:
    GKeys/s and the achieved bandwidth of its merge rounds."""
    import torch
    from paper_2505_18681_gb300 import inputs
    n = 100_000_000
    x = inputs.generate("uniform", n, torch.int32, seed=42, device=dev)
    y = torch.empty_like(x)
    p = evo.make_params(algo="merge", insertion_threshold=32, stream=stream)
    ms, recs, clocks, launches = _timed_with_profile(evo, lambda: evo.sort(x, out=y, params=p),
                                                     max(1, min(args.steps, 3)), 1, stream)
    passes = [r for r in recs if r["kind"] == "merge_pass"]
    ach = sum(r["bytes"] for r in passes) / 1e9 / (sum(r["ms"] for r in passes) * 1e-3) if passes else 0.0
    peak, src = measured_peaks()
    steps = max(1, min(args.steps, 3))
    return {"value": n / (ms * 1e-3) / 1e9, "unit": "GKeys/s", "ms_per_step": ms, "dtype": "i32",
            "config": {"workload": "mergesort of %d uniform int32 keys, insertion threshold 32" % n},
            "roofline": {"bound": "hbm", "kernel": "merge_pass", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak if peak else None, "traffic": None, "peak_source": src,
                         "rounds_per_sort": len(passes) // steps},
            "kernel_time_share": kernel_shares(recs), "clocks": clocks, "gpu_launches": launches}


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
    if args.workload == "segmented":
        # one rank per GPU under torchrun: each sorts its own share of the batch
        import torch.distributed as tdist
        ws, rank, local = dist_env()
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        if ws > 1:
            tdist.init_process_group("nccl", device_id=dev)
        res = leg_segmented(evo, args, torch.cuda.current_stream(), (lambda: tdist.barrier()) if ws > 1 else
                            (lambda: None), dev, nseg=args.segments, rank=rank, world=ws)
        if rank == 0:
            line.update(res)
            line["n_gpus"] = ws
            print(json.dumps(line), flush=True)
        if ws > 1:
            tdist.destroy_process_group()
        return
    if args.workload in ("floatpairs", "u32big", "small", "merge", "int32", "serving"):
        leg = {"floatpairs": leg_floatpairs, "u32big": leg_u32big, "small": leg_small, "merge": leg_merge,
               "int32": leg_int32, "serving": leg_serving}[args.workload]
        line.update(leg(evo, args, stream, lambda: None, torch.device("cuda")))
        print(json.dumps(line), flush=True)
        return
    if args.workload == "paper9":
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
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
