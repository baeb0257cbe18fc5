"""Continuous-batching sort server on one GPU.

Requests carry host (pinned) keys of int32, int64 or float64.  The loop:

* plans each request when it arrives: large ones (>= `big` keys) from a
  strided sample of their host keys (evosort_plan_host: the dispatcher's
  class and tuned parameters, with no device access), and computes what the
  request needs on the device: its keys plus the scratch of its sort
  (evosort_workspace_bytes / evosort_segmented_workspace_bytes);
* admits waiting requests in arrival order while the device has room for
  them: the HBM the server could use (free HBM as the CUDA driver reports
  it, plus what PyTorch's allocator holds unused, plus the server's own
  resident buffers), less a reserve, less what admitted but unfinished
  requests need;
* whenever one of its CUDA streams is idle, launches work on it: all admitted
  small requests of the oldest waiting dtype, packed into one batched
  segmented sort (one persistent launch sorts every request as its own
  segment), or one large request as a device-wide sort with its planned
  parameters;
* keeps one resident slot per stream (a key buffer, an offsets buffer and the
  sort's scratch, all passed to the library as caller memory), grown when a
  larger request comes and reused by every later launch on that stream, so
  the steady state allocates nothing;
* copies results back to host buffers on the same stream and marks requests
  done when the stream's event completes.

Requests that arrive while others are on the GPU are admitted and launched as
slots and memory free up, so their work overlaps on the device.  Each result
is the sort of that request alone: segments never mix, and the sort is
deterministic.  Latency is arrival to observed completion.

    python -m paper_2505_18681_gb300.serve --requests 300   # JSON summary line
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


class Request:
    __slots__ = ("rid", "keys", "out", "arrival", "admitted", "launched", "done", "n", "dtype", "nbytes",
                 "params", "need")

    def __init__(self, rid, keys: torch.Tensor, arrival: float):
        self.rid = rid
        self.keys = keys                      # pinned host input
        self.out = torch.empty_like(keys).pin_memory() if keys.numel() else torch.empty_like(keys)
        self.arrival = arrival
        self.admitted = self.launched = self.done = None
        self.n = keys.numel()
        self.dtype = keys.dtype
        self.nbytes = keys.numel() * keys.element_size()
        self.params = None                    # planned sort parameters (large requests)
        self.need = 0                         # device bytes while in flight


class Slot:
    """Device memory one stream keeps across launches: keys, offsets and the
    sort's scratch.  Grown on demand, never shrunk."""

    def __init__(self, dev):
        self.dev = dev
        self.keys = torch.empty(0, dtype=torch.uint8, device=dev)
        self.ws = torch.empty(0, dtype=torch.uint8, device=dev)
        self.offs = torch.empty(0, dtype=torch.int64, device=dev)

    @staticmethod
    def _grow(t, n, dtype, dev):
        if t.numel() < n:
            # geometric growth so a slowly rising size does not reallocate every time
            t = torch.empty(max(n, t.numel() + t.numel() // 2), dtype=dtype, device=dev)
        return t

    def key_view(self, n: int, dtype: torch.dtype) -> torch.Tensor:
        nb = n * torch.empty(0, dtype=dtype).element_size()
        self.keys = self._grow(self.keys, max(nb, 1), torch.uint8, self.dev)
        return self.keys[:nb].view(dtype)

    def workspace(self, nbytes: int) -> torch.Tensor:
        self.ws = self._grow(self.ws, max(nbytes, 1), torch.uint8, self.dev)
        return self.ws[:max(nbytes, 1)]

    def offsets(self, m: int) -> torch.Tensor:
        self.offs = self._grow(self.offs, m, torch.int64, self.dev)
        return self.offs[:m]

    def held(self) -> int:
        return self.keys.numel() + self.ws.numel() + self.offs.numel() * 8


class SortServer:
    def __init__(self, streams: int = 4, big: int = 1 << 20, batch_keys: int = 1 << 25,
                 reserve_bytes: int = 8 << 30, device: str = "cuda", use_table: str | None = None):
        import paper_2505_18681_gb300 as evo
        self.evo = evo
        evo.library()
        self.dev = torch.device(device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.slots = [Slot(self.dev) for _ in range(streams)]
        self.busy = [None] * streams          # (event, requests, pinned buffers) per stream
        self.big = big
        self.batch_keys = batch_keys
        self.reserve = reserve_bytes
        self.reserved = 0                     # bytes needed by admitted, unfinished requests
        self.waiting = collections.deque()    # arrived, not admitted
        self.admitted = collections.deque()   # admitted, not launched
        self.done = []
        self.launches = 0
        if use_table:
            evo.table_load(use_table)

    # -- memory accounting -------------------------------------------------
    def usable_bytes(self) -> int:
        """What the server could use: free HBM, PyTorch's unused cache and
        the server's own resident slots."""
        free, _ = torch.cuda.mem_get_info(self.dev)
        cached = torch.cuda.memory_reserved(self.dev) - torch.cuda.memory_allocated(self.dev)
        return free + cached + sum(s.held() for s in self.slots)

    def plan(self, r: Request) -> None:
        """Parameters and device bytes of a request (at arrival)."""
        evo = self.evo
        if r.n >= self.big:
            pd, _ = evo.plan_host(r.keys)
            r.params = pd
            r.need = r.nbytes + evo.workspace_bytes(r.n, r.dtype, **pd)
        else:
            # its share of a batch: keys, the segmented sort's scratch copy, an offset
            r.need = 2 * r.nbytes + 64

    # -- the loop ----------------------------------------------------------
    def submit(self, r: Request):
        self.plan(r)
        self.waiting.append(r)

    def _admit(self, now: float):
        usable = None
        while self.waiting:
            r = self.waiting[0]
            if self.reserved > 0:
                if usable is None:
                    usable = self.usable_bytes()
                if usable - self.reserve - self.reserved < r.need:
                    break   # wait for running work to release memory
            self.waiting.popleft()
            self.reserved += r.need
            r.admitted = now
            self.admitted.append(r)

    def _complete(self, now: float):
        for i, b in enumerate(self.busy):
            if b is not None and b[0].query():
                for r in b[1]:
                    r.done = now
                    self.reserved -= r.need
                    self.done.append(r)
                self.busy[i] = None

    def _launch(self, now: float):
        for i in range(len(self.streams)):
            if self.busy[i] is not None or not self.admitted:
                continue
            s = self.streams[i]
            head = self.admitted[0]
            keep = None
            if head.n >= self.big:
                self.admitted.popleft()
                batch = [head]
                self._launch_big(head, s, self.slots[i])
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
                keep = self._launch_batch(batch, s, self.slots[i])
            ev = torch.cuda.Event()
            ev.record(s)
            for r in batch:
                r.launched = now
            self.busy[i] = (ev, batch, keep)
            self.launches += 1

    def _launch_big(self, r: Request, s: torch.cuda.Stream, slot: Slot):
        evo = self.evo
        with torch.cuda.stream(s):
            d = slot.key_view(r.n, r.dtype)
            d.copy_(r.keys, non_blocking=True)
            ws = slot.workspace(evo.workspace_bytes(r.n, r.dtype, **r.params))
            # the plan came from the host sample: no device round trip here
            evo.sort(d, params=evo.make_params(stream=s, workspace=ws, **r.params))
            r.out.copy_(d, non_blocking=True)

    def _launch_batch(self, batch, s: torch.cuda.Stream, slot: Slot):
        evo = self.evo
        total = sum(r.n for r in batch)
        offs = torch.zeros(len(batch) + 1, dtype=torch.int64)
        offs[1:] = torch.cumsum(torch.tensor([r.n for r in batch], dtype=torch.int64), 0)
        offs = offs.pin_memory()
        with torch.cuda.stream(s):
            d = slot.key_view(total, batch[0].dtype)
            d_offs = slot.offsets(len(batch) + 1)
            d_offs.copy_(offs, non_blocking=True)
            o = 0
            for r in batch:
                if r.n:
                    d[o:o + r.n].copy_(r.keys, non_blocking=True)
                o += r.n
            ws = slot.workspace(evo.segmented_workspace_bytes(total, len(batch), batch[0].dtype))
            evo.segmented_sort(d, d_offs, params=evo.make_params(algo="radix", stream=s, workspace=ws))
            o = 0
            for r in batch:
                if r.n:
                    r.out.copy_(d[o:o + r.n], non_blocking=True)
                o += r.n
        return offs   # pinned: must outlive the copy, kept with the stream's work

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


def serve_mix(count: int, max_size: int = 100_000_000, streams: int = 4, load: float = 0.7, seed: int = 42,
              table: str | None = None, max_total: int | None = None) -> dict:
    """The serving measurement, on one server whose slots stay resident: the
    mix served with every request arriving at once, first to warm up (slot
    and pool growth, first launches) and then timed (capacity), then again
    with Poisson arrivals at `load` times that capacity; p50/p99 latency and
    keys/s of the Poisson run."""
    hi = size_upper_bound(count, 1000, max_size, max_total)
    reqs = make_requests(count, hi=max_size, seed=seed, max_total=max_total)
    srv = SortServer(streams=streams, use_table=table)

    def reset():
        for r in reqs:
            r.admitted = r.launched = r.done = None
        srv.done = []

    srv.run(reqs, [0.0] * len(reqs))   # warm-up
    reset()
    srv.run(reqs, [0.0] * len(reqs))
    cap = summarize(reqs, None, "saturated")
    lam = load * len(reqs) / cap["span_s"]
    g = torch.Generator().manual_seed(seed + 1)
    gaps = torch.empty(len(reqs), dtype=torch.float64).exponential_(lam, generator=g)
    arrivals = torch.cumsum(gaps, 0).tolist()
    reset()
    srv.launches = 0
    srv.run(reqs, arrivals)
    res = summarize(reqs, lam, "poisson")
    res["capacity_requests_per_s"] = len(reqs) / cap["span_s"]
    res["capacity_keys_per_s"] = cap["keys_per_s"]
    res["load"] = load
    res["launches"] = srv.launches
    res["size_range"] = [1000, hi]
    res["largest_request"] = max(r.n for r in reqs)
    res["dtypes"] = ["int32", "int64", "float64"]
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=300,
                    help="request count; sizes are log-uniform 1e3..1e8 (mean about 8.7e6 keys)")
    ap.add_argument("--max-size", type=int, default=100_000_000)
    ap.add_argument("--max-total", type=int, default=None, help="cap on the sum of request sizes")
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--load", type=float, default=0.7, help="arrival rate as a fraction of capacity")
    ap.add_argument("--seed", type=int, default=42)
    ap.add_argument("--table", default=None)
    a = ap.parse_args()
    print(json.dumps(serve_mix(a.requests, a.max_size, a.streams, a.load, a.seed, a.table, a.max_total)),
          flush=True)


if __name__ == "__main__":
    main()
