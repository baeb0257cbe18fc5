"""The continuous-batching server: every request's result equals the oracle's
sort of that request, and is the same when the request is served alone and
in the mix (tolerance: bit-exact)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def bits(t):
    a = t.numpy()
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def test_same_alone_and_in_the_mix():
    from paper_2505_18681_gb300 import serve
    reqs = serve.make_requests(48, lo=1000, hi=3_000_000, seed=7)
    g = torch.Generator().manual_seed(9)
    arrivals = torch.cumsum(torch.empty(len(reqs), dtype=torch.float64).exponential_(2000.0, generator=g), 0)
    srv = serve.SortServer(streams=3, big=1 << 20, batch_keys=1 << 22)
    srv.run(reqs, arrivals.tolist())
    assert all(r.done is not None for r in reqs)
    assert srv.launches < len(reqs)          # small requests were batched
    mixed = [r.out.clone() for r in reqs]
    for r, m in zip(reqs, mixed):
        assert np.array_equal(bits(m), bits(torch.from_numpy(oracle.radix_sort(r.keys.numpy()))))
    # each request alone through a fresh server
    for r, m in zip(reqs[:16], mixed[:16]):
        alone = serve.Request(r.rid, r.keys, 0.0)
        serve.SortServer(streams=1).run([alone], [0.0])
        assert torch.equal(alone.out.view(torch.uint8), m.view(torch.uint8))


def test_admission_waits_for_memory():
    """With a reserve larger than free memory, requests are still served one
    at a time (the loop always admits when nothing is running)."""
    from paper_2505_18681_gb300 import serve
    reqs = serve.make_requests(6, lo=1000, hi=20_000, seed=3)
    free, _ = torch.cuda.mem_get_info()
    srv = serve.SortServer(streams=2, reserve_bytes=free * 2)
    srv.run(reqs, [0.0] * len(reqs))
    for r in reqs:
        assert np.array_equal(bits(r.out), bits(torch.from_numpy(oracle.radix_sort(r.keys.numpy()))))
