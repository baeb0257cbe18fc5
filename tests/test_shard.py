"""Host logic of the segmented batch sharded over ranks (no data exchange):
the partition (every segment on exactly one rank, balanced loads), the
per-rank generation of a seeded batch, and a world_size-2 gloo run in which
each rank sorts its own share and the assembled result equals the oracle's
segmented sort of the whole batch.  In this CPU-only test the oracle stands
in for each rank's device call."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402  (the repository root is on the path only from here on)


def test_partition_covers_every_segment_once_and_balances():
    from paper_2505_18681_gb300 import inputs, shard
    lens = inputs.segment_lengths(10_000, 16, 1_000_000, seed=7)
    for world in (1, 2, 3, 8):
        owned, loads = shard.partition_segments(lens, world)
        flat = sorted(i for part in owned for i in part)
        assert flat == list(range(lens.numel()))
        assert sum(loads) == int(lens.sum())
        # longest-processing-time rule: the spread is at most one segment
        assert max(loads) - min(loads) <= int(lens.max())
        assert all(part == sorted(part) for part in owned)
    assert shard.partition_segments(lens, 4) == shard.partition_segments(lens, 4)
    with pytest.raises(ValueError):
        shard.partition_segments(lens, 0)


def test_rank_batches_are_the_global_batch_in_pieces():
    from paper_2505_18681_gb300 import inputs, shard
    lens = inputs.segment_lengths(700, 1, 5000, seed=2)
    lens[3] = 0
    keys, offs = inputs.segmented_keys(lens, torch.int32, seed=2)
    owned, _ = shard.partition_segments(lens, 3)
    out = torch.empty_like(keys)
    for part in owned:
        k, lo = shard.rank_batch(lens, part, torch.int32, seed=2)
        assert torch.equal(k, shard.gather_segments(keys, offs, part))
        assert int(lo[-1]) == k.numel()
        shard.scatter_segments(k, out, offs, part)
    assert torch.equal(out, keys)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as tdist
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2505_18681_gb300 import inputs, shard
    lens = inputs.segment_lengths(3_000, 16, 20_000, seed=5)
    owned, _ = shard.partition_segments(lens, world)
    mine = owned[rank]
    keys, lo = shard.rank_batch(lens, mine, torch.int64, seed=5)
    # this rank's share, sorted on its own (the oracle stands in for the
    # device call here); nothing is exchanged before the results are gathered
    local = oracle.segmented_sort(keys.numpy(), lo.numpy().astype(np.uint64))
    parts = [None] * world
    tdist.all_gather_object(parts, (mine, local))
    if rank == 0:
        full, offs = inputs.segmented_keys(lens, torch.int64, seed=5)
        expect = oracle.segmented_sort(full.numpy(), offs.numpy().astype(np.uint64))
        seen = [0] * lens.numel()
        res = torch.empty_like(full)
        for segs, arr in parts:
            for i in segs:
                seen[i] += 1
            shard.scatter_segments(torch.from_numpy(arr), res, offs, segs)
        out["once"] = all(c == 1 for c in seen)
        out["equal"] = bool(np.array_equal(res.numpy(), expect))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_ranks_sort_their_shares_into_the_oracle_result():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res["once"], "a segment was sorted by no rank or by two"
    assert res["equal"], "the assembled shards differ from the oracle's segmented sort"


# ---------------------------------------------------------------------------
# One array over several gloo ranks (sort_distributed), with the per-rank
# steps done on the CPU by the oracle: the exchange logic (range and
# histogram reductions, boundaries, run lengths, all-to-all) is what runs.
# ---------------------------------------------------------------------------
class _OracleOps:
    """Per-rank steps on CPU tensors: keys mapped to the order-preserving
    unsigned space of their integer type (sign bit flipped; descending:
    complemented), sorted by the oracle."""

    @staticmethod
    def _mapped(keys, descending):
        a = keys.numpy()
        u = a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)
        if a.dtype.kind == "i":
            u = u ^ (np.uint32(1 << 31) if a.dtype.itemsize == 4 else np.uint64(1 << 63))
        return ~u if descending else u

    def key_range(self, keys, descending):
        if keys.numel() == 0:
            return 2**64 - 1, 0
        m = self._mapped(keys, descending)
        return int(m.min()), int(m.max())

    def histogram(self, keys, base, shift, nbins, descending):
        m = self._mapped(keys, descending).astype(np.uint64)
        b = ((m - np.uint64(base)) >> np.uint64(shift)).astype(np.int64)
        return torch.from_numpy(np.bincount(np.minimum(b, nbins - 1), minlength=nbins).astype(np.int64))

    def sort(self, keys, values, descending):
        m = self._mapped(keys, descending)
        idx = np.arange(keys.numel(), dtype=np.uint32)
        _, perm = oracle.radix_sort(m, idx)
        k = torch.from_numpy(keys.numpy()[perm.astype(np.int64)].copy())
        v = None if values is None else torch.from_numpy(values.numpy()[perm.astype(np.int64)].copy())
        return k, v


def _dist_worker(rank, world, port, out, dtype_name, descending, pairs, n, dist_kind):
    import torch.distributed as tdist
    from paper_2505_18681_gb300 import shard
    tdist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    dtype = getattr(torch, dtype_name)
    g = torch.Generator().manual_seed(17)
    if dist_kind == "near_zero":
        full = torch.randint(-(1 << 20), 1 << 20, (n,), generator=g, dtype=torch.int64).to(dtype)
    elif dist_kind == "few":
        full = (torch.randint(0, 5, (n,), generator=g, dtype=torch.int64) * 1000 - 2000).to(dtype)
    else:
        info = torch.iinfo(dtype)
        full = torch.randint(info.min, info.max, (n,), generator=g, dtype=torch.int64).to(dtype)
    cuts = [n * r // world for r in range(world + 1)]
    cuts[1] = max(cuts[1] - 7, 0)   # uneven slices
    mine = full[cuts[rank]:cuts[rank + 1]].clone()
    vals = torch.arange(cuts[rank], cuts[rank + 1], dtype=torch.int64).to(torch.int32).view(torch.uint32) \
        if pairs else None
    k, v = shard.sort_distributed(mine, vals, descending=descending, ops=_OracleOps(), nbins=256)
    parts = [None] * world
    tdist.all_gather_object(parts, (k.numpy(), None if v is None else v.view(torch.int32).numpy()))
    if rank == 0:
        keys = np.concatenate([p[0] for p in parts])
        a = full.numpy()
        u = a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64) ^ \
            (np.uint32(1 << 31) if a.dtype.itemsize == 4 else np.uint64(1 << 63))
        order_key = ~u if descending else u
        _, perm = oracle.radix_sort(order_key, np.arange(n, dtype=np.uint32))
        out["keys"] = bool(np.array_equal(keys, a[perm.astype(np.int64)]))
        out["sizes"] = [len(p[0]) for p in parts]
        if pairs:
            vals_all = np.concatenate([p[1] for p in parts]).view(np.uint32)
            out["values"] = bool(np.array_equal(vals_all, perm))
    tdist.barrier()
    tdist.destroy_process_group()


@pytest.mark.parametrize("world,dtype_name,descending,pairs,dist_kind",
                         [(2, "int64", False, False, "near_zero"), (3, "int32", False, True, "uniform"),
                          (2, "int32", True, True, "few"), (3, "int64", True, False, "uniform")])
def test_one_array_over_gloo_ranks(world, dtype_name, descending, pairs, dist_kind):
    """The ranks' runs, concatenated in rank order, are the oracle's sort of
    the whole array (stable for key / value sorts: values are the global
    indices), and keys of both signs near zero still spread over the ranks."""
    n = 30_011
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_dist_worker, args=(world, port, out, dtype_name, descending, pairs, n, dist_kind), nprocs=world,
                 join=True)
        res = dict(out)
    assert res["keys"], "the ranks' runs differ from the oracle's sort of the whole array"
    if pairs:
        assert res["values"], "values are not the stable order of the keys"
    if dist_kind != "few":
        assert min(res["sizes"]) > n // world * 0.8, res["sizes"]


def test_rank_boundaries_split_into_equal_shares():
    from paper_2505_18681_gb300 import shard
    h = torch.tensor([5, 0, 5, 10, 0, 0, 20])
    assert shard.rank_boundaries(h, 2) == [0, 4, 7]
    assert shard.rank_boundaries(h, 4) == [0, 3, 4, 7, 7]   # shares 10, 10, 20, 0: bins are not split
    assert shard.rank_boundaries(torch.zeros(8, dtype=torch.int64), 3) == [0, 0, 0, 8]
    assert shard.shift_for(0, 4096) == 0 and shard.shift_for(4095, 4096) == 0 and shard.shift_for(4096, 4096) == 1
