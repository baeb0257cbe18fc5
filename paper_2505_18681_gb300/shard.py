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
owns their part of the key range.  That needs one exchange step (all-reduce
of the top-digit histogram to fix each rank's key range, an all-to-all of the
keys, then a local sort on each rank), which this module does not build.
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
