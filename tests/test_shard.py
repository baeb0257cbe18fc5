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
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res["once"], "a segment was sorted by no rank or by two"
    assert res["equal"], "the assembled shards differ from the oracle's segmented sort"
