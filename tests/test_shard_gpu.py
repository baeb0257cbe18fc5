"""The segmented batch sharded over ranks, on the GPU: each rank's share
(generated on its own) sorted with one batched call; the assembled result
equals the oracle's segmented sort of the whole batch.  The ranks run one
after the other in this process: no rank waits on another (there is no
exchange), so this is the multi-rank data path on one GPU."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_shards_assemble_to_the_oracle_result(world):
    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import inputs, shard
    evo.library()
    lens = inputs.segment_lengths(4_000, 16, 200_000, seed=11)
    full, offs = inputs.segmented_keys(lens, torch.int32, seed=11)
    expect = oracle.segmented_sort(full.numpy(), offs.numpy().astype(np.uint64))
    owned, loads = shard.partition_segments(lens, world)
    res = torch.empty_like(full)
    for part in owned:
        keys, lo = shard.rank_batch(lens, part, torch.int32, seed=11, device="cuda")
        shard.sort_rank_batch(keys, lo)
        evo.sync()
        shard.scatter_segments(keys.cpu(), res, offs, part)
    assert np.array_equal(res.numpy(), expect)


# ---------------------------------------------------------------------------
# One array over ranks (sort_distributed) with the library's GPU steps.
# ---------------------------------------------------------------------------
def _mapped_host(a, descending=False):
    """Order-preserving unsigned image of keys, from the oracle's total order."""
    if a.dtype.kind == "f":
        u = np.array([oracle.ordered_bits(int(x), a.dtype) for x in
                      a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)], dtype=np.uint64)
    else:
        u = a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64).astype(np.uint64)
        if a.dtype.kind == "i":
            u = u ^ np.uint64(1 << (8 * a.dtype.itemsize - 1))
    if descending:
        u = u ^ np.uint64((1 << (8 * a.dtype.itemsize)) - 1)
    return u


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float32, torch.float64], ids=str)
@pytest.mark.parametrize("descending", [False, True])
def test_key_range_and_range_histogram(dtype, descending):
    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import inputs, shard
    evo.library()
    x = inputs.generate("float_mix" if dtype.is_floating_point else "gaussian", 5003, dtype, seed=4,
                        device="cuda")
    m = _mapped_host(x.cpu().numpy(), descending)
    lo, hi = evo.key_range(x, descending)
    assert (lo, hi) == (int(m.min()), int(m.max()))
    shift = shard.shift_for(hi - lo, 1024)
    h = evo.range_histogram(x, lo, shift, 1024, descending).cpu().numpy()
    want = np.bincount(((m - np.uint64(lo)) >> np.uint64(shift)).astype(np.int64), minlength=1024)
    assert np.array_equal(h, want)
    e = torch.empty(0, dtype=dtype, device="cuda")
    assert evo.key_range(e) == (2**64 - 1, 0)


def _gpu_dist_worker(rank, world, port, out, dtype_name, pairs):
    import torch.distributed as tdist
    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import inputs, shard
    torch.cuda.set_device(0)
    evo.library()
    tdist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    dtype = getattr(torch, dtype_name)
    n = 3_000_017
    full = inputs.generate("gaussian", n, dtype, seed=21, device="cpu")
    cuts = [n * r // world for r in range(world + 1)]
    mine = full[cuts[rank]:cuts[rank + 1]].cuda()
    vals = torch.arange(cuts[rank], cuts[rank + 1], dtype=torch.int64).to(torch.int32).view(torch.uint32).cuda() \
        if pairs else None
    k, v = shard.sort_distributed(mine, vals)
    evo.sync()
    parts = [None] * world
    tdist.all_gather_object(parts, (k.cpu().numpy(), None if v is None else v.view(torch.int32).cpu().numpy()))
    if rank == 0:
        keys = np.concatenate([p[0] for p in parts])
        a = full.numpy()
        if pairs:
            wk, wv = oracle.radix_sort(a, np.arange(n, dtype=np.uint32))
            out["values"] = bool(np.array_equal(np.concatenate([p[1] for p in parts]).view(np.uint32), wv))
        else:
            wk = oracle.radix_sort(a)
        out["keys"] = bool(np.array_equal(keys, wk))
        out["sizes"] = [len(p[0]) for p in parts]
    tdist.barrier()
    tdist.destroy_process_group()


@pytest.mark.parametrize("dtype_name,pairs", [("int64", False), ("int32", True)])
def test_one_array_over_two_ranks_on_one_gpu(dtype_name, pairs):
    """Two gloo ranks share the GPU (no kernel of one waits on the other: the
    collectives run on the host); Gaussian keys of both signs spread evenly
    over the ranks through the range-based bins."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_gpu_dist_worker, args=(2, port, out, dtype_name, pairs), nprocs=2, join=True)
        res = dict(out)
    assert res["keys"]
    if pairs:
        assert res["values"]
    assert min(res["sizes"]) > 3_000_017 // 2 * 0.9, res["sizes"]
