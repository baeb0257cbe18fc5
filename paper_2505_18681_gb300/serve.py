"""Continuous-batching sort server on one GPU.

Requests carry host (pinned) keys of int32, int64 or float64.  The loop:

* admits waiting requests in arrival order while the device has room for
  them: free HBM (free as the CUDA driver reports it, plus what PyTorch's allocator holds unused),
  less a reserve, less what admitted but unfinished requests have reserved;
* whenever one of its CUDA streams is idle, launches work on it: all admitted
  small requests of the oldest waiting dtype, packed into one batched
  segmented sort (one persistent launch sorts every request as its own
  segment), or one large request (>= `big` keys) as a device-wide radix sort
  with the dispatcher's parameters;
* copies results back to host buffers on the same stream and marks requests
  done when the stream's event completes.

Requests that arrive while others are on the GPU are admitted and launched as
slots and memory free up, so their work overlaps on the device.  Each result
is the sort of that request alone: segments never mix, and the sort is
deterministic.  Latency is arrival to observed completion.

    python -m paper_2505_18681_gb300.serve --requests 10000   # JSON summary line
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import statistics
import time

import torch

from . import inputs

DTYPES = {"int32": torch.int32, "int64": torch.int64, "float64": torch.float64}


class Request:
    __slots__ = ("rid", "keys", "out", "arrival", "admitted", "launched", "done", "n", "dtype", "nbytes")

    def __init__(self, rid, keys: torch.Tensor, arrival: float):
        self.rid = rid
        self.keys = keys                      # pinned host input
        self.out = torch.empty_like(keys).pin_memory() if keys.numel() else torch.empty_like(keys)
        self.arrival = arrival
        self.admitted = self.launched = self.done = None
        self.n = keys.numel()
        self.dtype = keys.dtype
        self.nbytes = keys.numel() * keys.element_size()


class SortServer:
    def __init__(self, streams: int = 4, big: int = 1 << 20, batch_keys: int = 1 << 25,
                 reserve_bytes: int = 8 << 30, device: str = "cuda", use_table: str | None = None):
        import paper_2505_18681_gb300 as evo
        self.evo = evo
        evo.library()
        self.dev = torch.device(device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.busy = [None] * streams          # (event, requests, buffers) per stream
        self.big = big
        self.batch_keys = batch_keys
        self.reserve = reserve_bytes
        self.reserved = 0                     # bytes held by admitted, unfinished requests
        self.pending = 0                      # of which not yet allocated (admitted, not launched)
        self.waiting = collections.deque()    # arrived, not admitted
        self.admitted = collections.deque()   # admitted, not launched
        self.done = []
        self.launches = 0
        if use_table:
            evo.table_load(use_table)

    # -- memory accounting -------------------------------------------------
    def free_bytes(self) -> int:
        free, _ = torch.cuda.mem_get_info(self.dev)
        cached = torch.cuda.memory_reserved(self.dev) - torch.cuda.memory_allocated(self.dev)
        return free + cached

    @staticmethod
    def need_bytes(r: Request) -> int:
        # device copy of the keys plus scratch of about the same size
        return 2 * r.nbytes + (1 << 20)

    # -- the loop ----------------------------------------------------------
    def submit(self, r: Request):
        self.waiting.append(r)

    def _admit(self, now: float):
        free = None
        while self.waiting:
            r = self.waiting[0]
            need = self.need_bytes(r)
            if self.reserved > 0:
                if free is None:
                    free = self.free_bytes()
                if free - self.pending - self.reserve < need:
                    break   # wait for running work to release memory
            self.waiting.popleft()
            self.reserved += need
            self.pending += need
            r.admitted = now
            self.admitted.append(r)

    def _complete(self, now: float):
        for i, b in enumerate(self.busy):
            if b is not None and b[0].query():
                for r in b[1]:
                    r.done = now
                    self.reserved -= self.need_bytes(r)
                    self.done.append(r)
                self.busy[i] = None

    def _launch(self, now: float):
        for i in range(len(self.streams)):
            if self.busy[i] is not None or not self.admitted:
                continue
            s = self.streams[i]
            head = self.admitted[0]
            if head.n >= self.big:
                self.admitted.popleft()
                batch = [head]
                bufs = self._launch_big(head, s)
            else:
                # all admitted small requests of the head's dtype, up to batch_keys keys
                batch, rest, total = [], collections.deque(), 0
                while self.admitted:
                    r = self.admitted.popleft()
                    if r.n < self.big and r.dtype == head.dtype and (total + r.n <= self.batch_keys or not batch):
                        batch.append(r)
                        total += r.n
                    else:
                        rest.append(r)
                self.admitted = rest
                bufs = self._launch_batch(batch, s)
            ev = torch.cuda.Event()
            ev.record(s)
            for r in batch:
                r.launched = now
                self.pending -= self.need_bytes(r)
            self.busy[i] = (ev, batch, bufs)
            self.launches += 1

    def _launch_big(self, r: Request, s: torch.cuda.Stream):
        with torch.cuda.stream(s):
            d = torch.empty(r.n, dtype=r.dtype, device=self.dev)
            d.copy_(r.keys, non_blocking=True)
            # the dispatcher would sample the keys on the device, a synchronous
            # read that would stall this loop; large requests take the radix path
            self.evo.sort(d, algo="radix", stream=s)
            r.out.copy_(d, non_blocking=True)
        return (d,)

    def _launch_batch(self, batch, s: torch.cuda.Stream):
        total = sum(r.n for r in batch)
        offs = torch.zeros(len(batch) + 1, dtype=torch.int64)
        offs[1:] = torch.cumsum(torch.tensor([r.n for r in batch], dtype=torch.int64), 0)
        offs = offs.pin_memory()
        with torch.cuda.stream(s):
            d = torch.empty(max(total, 1), dtype=batch[0].dtype, device=self.dev)[:total]
            d_offs = offs.to(self.dev, non_blocking=True)
            o = 0
            for r in batch:
                if r.n:
                    d[o:o + r.n].copy_(r.keys, non_blocking=True)
                o += r.n
            self.evo.segmented_sort(d, d_offs, stream=s)
            o = 0
            for r in batch:
                if r.n:
                    r.out.copy_(d[o:o + r.n], non_blocking=True)
                o += r.n
        return (d, d_offs, offs)

    def step(self, now: float):
        self._complete(now)
        self._admit(now)
        self._launch(now)

    def idle(self) -> bool:
        return not self.waiting and not self.admitted and all(b is None for b in self.busy)

    def run(self, requests, arrivals):
        """Feeds `requests` at wall-clock offsets `arrivals` (seconds from the
        start) and runs the loop until all are done.  Returns the requests."""
        order = sorted(range(len(requests)), key=lambda k: arrivals[k])
        t0 = time.perf_counter()
        k = 0
        while k < len(order) or not self.idle():
            now = time.perf_counter() - t0
            while k < len(order) and arrivals[order[k]] <= now:
                r = requests[order[k]]
                r.arrival = arrivals[order[k]]
                self.submit(r)
                k += 1
            self.step(now)
        for s in self.streams:
            s.synchronize()
        self.evo.sync()
        return requests


def size_upper_bound(count: int, lo: int, hi: int, max_total: int | None) -> int:
    """Largest upper size bound <= hi whose expected total, count times the
    mean of a log-uniform size on [lo, hi'], stays within max_total."""
    def mean(h):
        return (h - lo) / math.log(h / lo) if h > lo else lo
    if max_total is None or count * mean(hi) <= max_total:
        return hi
    a, b = lo, hi
    for _ in range(100):
        m = (a + b) / 2
        if count * mean(m) <= max_total:
            a = m
        else:
            b = m
    return int(a)


def make_requests(count: int, lo: int = 1000, hi: int = 100_000_000, seed: int = 42, max_total: int | None = None):
    """Seeded request mix: sizes floor(exp(U(ln lo, ln hi))), dtype uniform over
    int32 / int64 / float64, distributions as in the sort workloads.  With
    max_total the upper size bound is lowered so the expected total fits."""
    hi = size_upper_bound(count, lo, hi, max_total)
    g = torch.Generator().manual_seed(seed)
    u = torch.rand(count, generator=g, dtype=torch.float64)
    sizes = torch.floor(torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).to(torch.int64)
    kinds = torch.randint(0, 3, (count,), generator=g)
    dists = ["uniform", "gaussian", "sorted", "reverse", "nearly_sorted", "distinct16", "zipf", "equal",
             "uniform1000"]
    dpick = torch.randint(0, len(dists), (count,), generator=g)
    reqs = []
    for i in range(count):
        dt = [torch.int32, torch.int64, torch.float64][int(kinds[i])]
        dist = "float_mix" if dt == torch.float64 else dists[int(dpick[i])]
        x = inputs.generate(dist, int(sizes[i]), dt, seed=seed + i, device="cuda").cpu().pin_memory()
        reqs.append(Request(i, x, 0.0))
    return reqs


def summarize(reqs, lam, label):
    lat = sorted((r.done - r.arrival) * 1e3 for r in reqs)
    keys = sum(r.n for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    q = lambda p: lat[min(len(lat) - 1, int(p * len(lat)))]
    return {"label": label, "requests": len(reqs), "keys": keys, "lambda_per_s": lam,
            "p50_ms": q(0.50), "p99_ms": q(0.99), "mean_ms": statistics.fmean(lat),
            "keys_per_s": keys / span, "span_s": span}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=10_000)
    ap.add_argument("--max-size", type=int, default=100_000_000)
    ap.add_argument("--max-total", type=int, default=None, help="cap on the sum of request sizes")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--load", type=float, default=0.7, help="arrival rate as a fraction of capacity")
    ap.add_argument("--seed", type=int, default=42)
    ap.add_argument("--table", default=None)
    a = ap.parse_args()
    hi = size_upper_bound(a.requests, 1000, a.max_size, a.max_total)
    reqs = make_requests(a.requests, hi=a.max_size, seed=a.seed, max_total=a.max_total)
    srv = SortServer(streams=a.streams, use_table=a.table)
    # capacity: everything arrives at once
    srv.run(reqs, [0.0] * len(reqs))
    cap = summarize(reqs, None, "saturated")
    lam = a.load * len(reqs) / cap["span_s"]
    g = torch.Generator().manual_seed(a.seed + 1)
    gaps = torch.empty(len(reqs), dtype=torch.float64).exponential_(lam, generator=g)
    arrivals = torch.cumsum(gaps, 0).tolist()
    for r in reqs:
        r.done = None
    srv = SortServer(streams=a.streams, use_table=a.table)
    srv.run(reqs, arrivals)
    res = summarize(reqs, lam, "poisson")
    res["capacity_requests_per_s"] = len(reqs) / cap["span_s"]
    res["capacity_keys_per_s"] = cap["keys_per_s"]
    res["launches"] = srv.launches
    res["size_range"] = [1000, hi]
    res["dtypes"] = ["int32", "int64", "float64"]
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
