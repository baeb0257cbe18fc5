"""evosort_release: the scratch a sort leaves reserved in the device's
stream-ordered pool goes back to the CUDA driver, and sorts after the release
still match the CPU oracle.  (Memory management of this library; the paper
has no counterpart.)"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    evo.table_clear()
    return evo


def test_release_returns_pooled_scratch(evo):
    from paper_2505_18681_gb300 import inputs
    n = 100_000_000
    x = inputs.generate("uniform", n, torch.int64, seed=3, device="cuda")
    y = torch.empty_like(x)
    evo.sort(x, out=y)
    evo.sync()
    need = evo.workspace_bytes(n, torch.int64)
    assert need > 500_000_000
    free0, _ = torch.cuda.mem_get_info()
    evo.release()
    free1, _ = torch.cuda.mem_get_info()
    # the sort's scratch was back in the pool (freed in stream order at its
    # end); trimming the pool hands at least that much to the CUDA driver
    assert free1 - free0 >= need // 2, (free0, free1, need)
    del x, y
    torch.cuda.empty_cache()
    # later sorts reserve again and are still exact
    for n2 in (1000, 100_000, 3_000_001):
        a = inputs.generate("gaussian", n2, torch.int64, seed=n2, device="cuda")
        b = torch.empty_like(a)
        evo.sort(a, out=b)
        evo.sync()
        assert np.array_equal(b.cpu().numpy(), oracle.radix_sort(a.cpu().numpy()))
    evo.release()
    evo.release()   # nothing left to trim: still fine
