"""Batched segmented sort over several GPUs, one process per GPU.

The segments of a batch are independent (each is sorted on its own), so a
batch shards across ranks by whole segments: no key ever has to reach
another rank, and there is no collective on the data path.  Segments are
assigned longest first, each to the rank with the least work so far (the
longest-processing-time rule; ties go to the lower rank), which keeps every
rank's key count within one segment of the mean.  Each rank gathers its
segments into one contiguous local batch, sorts it with one batched call
(evosort_segmented_sort) and can write the results back to the segments'
global positions.

A single array does not shard this way: its keys must move to the rank that
owns their part of the key range.  sort_distributed (below) does that with
one exchange step: two reductions fix the global key range and a histogram
of it, the ranks split the histogram into equal shares, and one all-to-all
moves every key to the rank owning its share before a local sort.
"""
from __future__ import annotations

import heapq

import torch

from . import inputs


def partition_segments(lengths, world: int):
    """Segment ids of each rank (ascending) and each rank's key count.

    ``lengths``: segment lengths (sequence or 1-D tensor), ``world``: ranks.
    Longest segment first, each to the rank with the fewest keys so far;
    equal lengths in segment order, equal loads to the lower rank."""
    if world < 1:
        raise ValueError("world must be at least 1")
    lens = [int(v) for v in (lengths.tolist() if isinstance(lengths, torch.Tensor) else lengths)]
    order = sorted(range(len(lens)), key=lambda i: (-lens[i], i))
    heap = [(0, r) for r in range(world)]
    owned = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        owned[r].append(i)
        heapq.heappush(heap, (load + lens[i], r))
    loads = [0] * world
    for r in range(world):
        owned[r].sort()
        loads[r] = sum(lens[i] for i in owned[r])
    return owned, loads


def local_offsets(lengths, seg_ids) -> torch.Tensor:
    """Offsets (int64, len(seg_ids) + 1) of the local batch made of the
    given segments, concatenated in the given order."""
    lens = torch.as_tensor(lengths, dtype=torch.int64).cpu()
    sel = lens[torch.as_tensor(seg_ids, dtype=torch.int64)] if len(seg_ids) else torch.zeros(0, dtype=torch.int64)
    offs = torch.zeros(sel.numel() + 1, dtype=torch.int64)
    offs[1:] = torch.cumsum(sel, 0)
    return offs


def gather_segments(keys: torch.Tensor, offsets: torch.Tensor, seg_ids) -> torch.Tensor:
    """The keys of the given segments of a global batch, concatenated (on the
    keys' device)."""
    offs = offsets.cpu().tolist()
    parts = [keys[offs[i]:offs[i + 1]] for i in seg_ids]
    return torch.cat(parts) if parts else keys[:0].clone()


def scatter_segments(local: torch.Tensor, out: torch.Tensor, offsets: torch.Tensor, seg_ids) -> None:
    """Writes a local batch's segments back to their global positions in
    ``out`` (the inverse of gather_segments)."""
    offs = offsets.cpu().tolist()
    o = 0
    for i in seg_ids:
        m = offs[i + 1] - offs[i]
        out[offs[i]:offs[i + 1]] = local[o:o + m]
        o += m


def rank_batch(lengths, seg_ids, dtype=torch.int32, seed: int = 42, device="cpu"):
    """This rank's local batch of a seeded global batch, generated directly:
    the keys of the given segments exactly as inputs.segmented_keys would
    produce them for the whole batch (the generator is counter-based on the
    global position), and the local offsets."""
    lens = torch.as_tensor(lengths, dtype=torch.int64).cpu()
    g_offs = torch.zeros(lens.numel() + 1, dtype=torch.int64)
    g_offs[1:] = torch.cumsum(lens, 0)
    l_offs = local_offsets(lens, seg_ids)
    total = int(l_offs[-1])
    keys = torch.empty(total, dtype=dtype, device=device)
    o = 0
    for i in seg_ids:
        a, b = int(g_offs[i]), int(g_offs[i + 1])
        if b > a:
            keys[o:o + (b - a)] = inputs.segmented_keys_range(lens, a, b, dtype, seed=seed, device=device)
        o += b - a
    return keys, l_offs


def sort_rank_batch(keys: torch.Tensor, local_offs: torch.Tensor, **params) -> torch.Tensor:
    """Sorts this rank's local batch in place with one batched call."""
    from . import segmented_sort
    return segmented_sort(keys, local_offs.to(keys.device), **params)


# ---------------------------------------------------------------------------
# One array over several ranks.  Each rank holds a slice; on return rank r
# holds a sorted run and every key of rank r precedes (in the sort's order)
# every key of rank r + 1.  Steps: the global key range (two reductions of
# the slices' smallest and largest keys); a histogram of every slice over
# NBINS equal parts of that range, summed over the ranks; bin boundaries
# between ranks at the prefix sums closest to equal shares; each slice
# sorted locally, so the keys it sends to a rank are one contiguous run whose
# length its own histogram gives; one exchange of the run lengths and one of
# the keys (and values); a local sort of what arrived.  Equal keys fall in
# one bin, so a value held by more than a rank's share of the keys is not
# split (that rank receives all of it).  Key / value sorts are stable in
# (rank, index within the slice) order: runs arrive in rank order and both
# local sorts are stable.
# ---------------------------------------------------------------------------
NBINS = 4096


class DeviceOps:
    """The per-rank steps on the slice's GPU, through the library."""

    def key_range(self, keys, descending):
        from . import key_range
        return key_range(keys, descending)

    def histogram(self, keys, base, shift, nbins, descending):
        from . import range_histogram
        return range_histogram(keys, base, shift, nbins, descending).cpu()

    def sort(self, keys, values, descending):
        from . import sort, sort_pairs
        if values is None:
            return sort(keys, descending=descending), None
        return sort_pairs(keys, values, descending=descending)


def shift_for(span: int, nbins: int) -> int:
    """Smallest shift with span >> shift < nbins (nbins a power of two)."""
    return max(0, span.bit_length() - (nbins.bit_length() - 1))


def rank_boundaries(hist, world: int):
    """First bin of each rank (and nbins at the end): rank r owns the bins
    from the first one at which the keys before it reach r / world of all
    keys."""
    h = torch.as_tensor(hist, dtype=torch.int64).cpu()
    before = torch.zeros(h.numel() + 1, dtype=torch.int64)
    before[1:] = torch.cumsum(h, 0)
    total = int(before[-1])
    bounds = [0]
    for r in range(1, world):
        want = -(-total * r // world)   # ceil
        bounds.append(int(torch.searchsorted(before, torch.tensor(want), right=False)))
    bounds.append(h.numel())
    for r in range(1, world + 1):   # non-decreasing, within [0, nbins]
        bounds[r] = min(max(bounds[r], bounds[r - 1]), h.numel())
    return bounds


def _signed(x: int) -> int:
    """Unsigned 64-bit key as the int64 of the same order (top bit flipped)."""
    y = x ^ (1 << 63)
    return y - (1 << 64) if y >= (1 << 63) else y


def _unsigned(y: int) -> int:
    return (y + (1 << 64) if y < 0 else y) ^ (1 << 63)


def _wire(t):
    """Transport view of keys: signed integers of the same width (the
    collectives need no unsigned types); floats travel as they are."""
    if t.dtype == torch.uint32:
        return t.view(torch.int32)
    if t.dtype == torch.uint64:
        return t.view(torch.int64)
    return t


def sort_distributed(keys, values=None, *, descending=False, group=None, ops=None, nbins=NBINS):
    """Sorts the union of the ranks' key slices (1-D, same dtype on every
    rank) across the ranks; returns this rank's sorted run (and its values:
    uint32, one per key, moved with their keys).  Collective: every rank of
    the group calls it."""
    import torch.distributed as dist
    ops = ops or DeviceOps()
    world = dist.get_world_size(group)
    comm = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else \
        torch.device("cpu")
    # global key range
    lo, hi = ops.key_range(keys, descending)
    rlo = torch.tensor([_signed(lo)], dtype=torch.int64, device=comm)
    rhi = torch.tensor([_signed(hi)], dtype=torch.int64, device=comm)
    dist.all_reduce(rlo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(rhi, op=dist.ReduceOp.MAX, group=group)
    glo, ghi = _unsigned(int(rlo[0])), _unsigned(int(rhi[0]))
    if ghi < glo:   # no keys on any rank
        return keys, values
    shift = shift_for(ghi - glo, nbins)
    # slice histograms, summed over the ranks; boundaries between ranks
    local = ops.histogram(keys, glo, shift, nbins, descending).to(torch.int64)
    glob = local.to(comm).clone()
    dist.all_reduce(glob, group=group)
    bounds = rank_boundaries(glob, world)
    # local sort; the run for rank r is the slice's keys in bins [b_r, b_{r+1})
    keys, values = ops.sort(keys, values, descending)
    before = torch.zeros(nbins + 1, dtype=torch.int64)
    before[1:] = torch.cumsum(local.cpu(), 0)
    send = [int(before[bounds[r + 1]] - before[bounds[r]]) for r in range(world)]
    sc = torch.tensor(send, dtype=torch.int64, device=comm)
    rc = torch.empty(world, dtype=torch.int64, device=comm)
    dist.all_to_all_single(rc, sc, group=group)
    recv = [int(v) for v in rc.tolist()]
    wk = _wire(keys).to(comm)
    out = torch.empty(sum(recv), dtype=wk.dtype, device=comm)
    dist.all_to_all_single(out, wk, recv, send, group=group)
    got = out.to(keys.device).view(keys.dtype)
    gv = None
    if values is not None:
        wv = values.view(torch.int32).to(comm)
        vo = torch.empty(sum(recv), dtype=torch.int32, device=comm)
        dist.all_to_all_single(vo, wv, recv, send, group=group)
        gv = vo.to(values.device).view(values.dtype)
    if got.numel() > 1:
        got, gv = ops.sort(got, gv, descending)
    return got, gv
