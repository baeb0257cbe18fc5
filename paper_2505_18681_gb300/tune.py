"""Builds the tuned-parameter table with the genetic algorithm (Algorithm 2).

For each distribution class the dispatcher tells apart, the GA runs on a
seeded sample of a representative workload of that class, on the GPU, and
the winning parameters go into the table under (dtype, floor(log2 n), class).
Candidates are verified on the device (sortedness and a multiset fingerprint
of the input); no CPU code takes part.  The paper tunes per array size with a
population of 30 over 10 generations (Section 4.2); so does this script, per
class as well.

    python -m paper_2505_18681_gb300.tune --dtype int64 --n 268435456 \\
        --out paper_2505_18681_gb300/tuned/gb300_int64.txt
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
        t0 = time.time()
        best, ms, log = evo.tune(x, population=population, generations=generations, reps=reps, seed=seed)
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
    a = ap.parse_args()
    evo.library()
    if os.path.exists(a.out):
        evo.table_load(a.out)
    tune_table(getattr(torch, a.dtype), a.n, a.classes.split(","), a.seed, a.population, a.generations, a.reps,
               a.log)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    evo.table_save(a.out)


if __name__ == "__main__":
    main()
