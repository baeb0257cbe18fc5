"""Builds the tuned-parameter table with the genetic algorithm (Algorithm 2).

For each distribution class the dispatcher tells apart, the GA runs on a
seeded sample of a representative workload of that class, on the GPU, and
the winning parameters go into the table under (dtype, floor(log2 n), class).
Every candidate's output is compared bit for bit with a reference sort of the
same sample made once before the search by a different kernel (the staged
radix tile with fixed parameters); no CPU code takes part.  The paper tunes
per array size with a population of 30 over 10 generations (Section 4.2); so
does this script, per class as well.  With --mode segmented the GA tunes the
batched segmented sort's tier cut-overs on a batch of log-uniform segment
lengths and stores them under the 'segmented' class.

    python -m paper_2505_18681_gb300.tune --dtype int64 --n 268435456 \\
        --out paper_2505_18681_gb300/tuned/gb300_int64.txt
    python -m paper_2505_18681_gb300.tune --mode segmented --dtype int32 --segments 10000 \\
        --out paper_2505_18681_gb300/tuned/gb300_int32.txt
"""
from __future__ import annotations

import argparse
import json
import os
import time

import torch

from . import inputs

# representative workload of each class (dispatcher classes, see evosort.h)
REPRESENTATIVE = {
    "random": "uniform",
    "skewed": "gaussian",
    "narrow": "zipf",
    "narrow16": "uniform1000",
    "few": "distinct16",
    "sorted": "nearly_sorted",
    "reverse": "reverse",
    "constant": "equal",
}


def bucket(n: int) -> int:
    return max(n, 1).bit_length() - 1


def time_params(x, params: dict, reps: int) -> float:
    """Best-of-reps device time (ms) of one sort of x with the given parameters."""
    import paper_2505_18681_gb300 as evo
    out = torch.empty_like(x)
    s = torch.cuda.current_stream()
    evo.sort(x, out=out, **params)
    best = float("inf")
    for _ in range(max(reps, 1)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        evo.sort(x, out=out, **params)
        e1.record(s)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    evo.sync()
    return best


def tune_table(dtype=torch.int64, n=1 << 28, classes=None, seed=42, population=30, generations=10, reps=3,
               log_path=None, verbose=True):
    import paper_2505_18681_gb300 as evo
    classes = classes or list(REPRESENTATIVE)
    results = {}
    for cls in classes:
        dist = REPRESENTATIVE[cls]
        x = inputs.generate(dist, n, dtype, seed=seed, device="cuda")
        got = evo.classify(x)
        # the table's current entry for this class (or the built-in defaults)
        incumbent, _ = evo.plan(x)
        # the reference every candidate must equal: the staged tile, fixed
        # parameters (a kernel the search mostly does not use)
        ref = torch.empty_like(x)
        evo.sort(x, out=ref, algo="radix", pass_kernel=1, rank_mode=3, digit_bits=8, small_cap=1)
        evo.sync()
        t0 = time.time()
        best, ms, log = evo.tune(x, expected=ref, population=population, generations=generations, reps=reps,
                                 seed=seed)
        del ref
        dt = time.time() - t0
        # a search can miss a corner the previous one found: both are timed
        # the same way and the faster one is kept
        t_new = time_params(x, best, reps)
        t_old = time_params(x, incumbent, reps)
        kept = "search"
        if t_old < t_new:
            best, ms, kept = incumbent, t_old, "incumbent"
        else:
            ms = t_new
        evo.table_set(dtype, bucket(n), cls, best, ms)
        results[cls] = {"distribution": dist, "sampled_class": got, "best": best, "best_ms": ms, "kept": kept,
                        "search_ms": t_new, "incumbent": incumbent, "incumbent_ms": t_old,
                        "tune_seconds": round(dt, 1), "log": log}
        if verbose:
            print("%-9s %-14s class=%-9s best %.3f ms %s kept=%s (search %.3f, incumbent %.3f; %.0f s)"
                  % (cls, dist, got, ms, best, kept, t_new, t_old, dt), flush=True)
        del x
        torch.cuda.empty_cache()
    if log_path:
        with open(log_path, "w") as f:
            json.dump({"dtype": str(dtype), "n": n, "bucket": bucket(n), "population": population,
                       "generations": generations, "reps": reps, "seed": seed, "classes": results}, f, indent=1)
    return results


def tune_segmented(dtype=torch.int32, nseg=10_000, lo=16, hi=1_000_000, seed=42, population=30, generations=10,
                   reps=3, verbose=True):
    """GA over the segmented sort's tier cut-overs (warp tier, block tier,
    giant segments) and the block tier's insertion threshold, on a batch of
    nseg segments with log-uniform lengths lo..hi (half uniform, half nearly
    sorted keys).  Fitness: the median device time of the batched sort; a
    candidate whose output differs from the reference batch sort (made once
    with the built-in cut-overs) fails."""
    import paper_2505_18681_gb300 as evo
    lens = inputs.segment_lengths(nseg, lo, hi, seed=seed)
    keys, offs = inputs.segmented_keys(lens, dtype, seed=seed, device="cuda")
    d_offs = offs.to("cuda")
    total = keys.numel()
    ref = keys.clone()
    evo.segmented_sort(ref, d_offs, algo="radix")
    evo.sync()
    work = torch.empty_like(keys)
    s = torch.cuda.current_stream()

    def fitness(p, _best):
        params = evo.make_params(stream=s, **p)
        ts = []
        for _ in range(max(reps, 1)):
            work.copy_(keys)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            try:
                evo.segmented_sort(work, d_offs, params=params)
            except evo.EvoSortError:
                return -1.0
            e1.record(s)
            try:
                evo.sync(s)
            except evo.EvoSortError:
                return -1.0
            ts.append(e0.elapsed_time(e1))
            if not torch.equal(work, ref):
                return -1.0
        ts.sort()
        return ts[len(ts) // 2]

    t0 = time.time()
    best, ms, log = evo.ga_search(fitness, key_bytes=keys.element_size(), mode=1, population=population,
                                  generations=generations, seed=seed)
    evo.table_set(dtype, bucket(total), "segmented", best, ms)
    if verbose:
        print("segmented %d segments, %d keys: best %.3f ms %s (%.0f s)" % (nseg, total, ms, best,
                                                                             time.time() - t0), flush=True)
    return {"segments": nseg, "total": total, "best": best, "best_ms": ms, "log": log,
            "defaults_ms": log[0]["best_ms"] if log else None}


def main():
    import paper_2505_18681_gb300 as evo
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="int64")
    ap.add_argument("--n", type=int, default=1 << 28)
    ap.add_argument("--classes", default=",".join(REPRESENTATIVE))
    ap.add_argument("--population", type=int, default=30)
    ap.add_argument("--generations", type=int, default=10)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=42)
    ap.add_argument("--out", required=True)
    ap.add_argument("--log", default=None)
    ap.add_argument("--mode", default="array", choices=["array", "segmented"])
    ap.add_argument("--segments", type=int, default=10_000)
    a = ap.parse_args()
    evo.library()
    if os.path.exists(a.out):
        evo.table_load(a.out)
    if a.mode == "segmented":
        res = tune_segmented(getattr(torch, a.dtype), a.segments, seed=a.seed, population=a.population,
                             generations=a.generations, reps=a.reps)
        if a.log:
            with open(a.log, "w") as f:
                json.dump(res, f, indent=1)
    else:
        tune_table(getattr(torch, a.dtype), a.n, a.classes.split(","), a.seed, a.population, a.generations,
                   a.reps, a.log)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    evo.table_save(a.out)


if __name__ == "__main__":
    main()
