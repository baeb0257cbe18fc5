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
