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
    # one request far above the batching cut-over (3.2e7 keys): planned from
    # its host sample, sorted in its stream's resident slot
    from paper_2505_18681_gb300 import inputs
    xb = inputs.generate("gaussian", 32_000_017, torch.int64, seed=5, device="cuda").cpu().pin_memory()
    reqs.insert(20, serve.Request(len(reqs), xb, 0.0))
    g = torch.Generator().manual_seed(9)
    arrivals = torch.cumsum(torch.empty(len(reqs), dtype=torch.float64).exponential_(2000.0, generator=g), 0)
    srv = serve.SortServer(streams=3, big=1 << 20, batch_keys=1 << 22)
    srv.run(reqs, arrivals.tolist())
    assert all(r.done is not None for r in reqs)
    assert srv.launches < len(reqs)          # small requests were batched
    assert max(r.n for r in reqs) > 30_000_000
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


def test_resident_slots_are_reused():
    """Launches reuse their stream's resident slot: once every slot holds
    enough for the largest launch, serving a mix allocates nothing more."""
    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import serve
    reqs = serve.make_requests(12, lo=1000, hi=4_000_000, seed=13)
    srv = serve.SortServer(streams=2, big=1 << 20, batch_keys=1 << 22)
    most = max(r.n for r in reqs) + (1 << 22)
    for slot in srv.slots:
        slot.key_view(most, torch.int64)
        slot.offsets(len(reqs) + 1)
        slot.workspace(max(evo.workspace_bytes(most, torch.int64), evo.segmented_workspace_bytes(most, len(reqs),
                                                                                               torch.int64)))
    held = [s.held() for s in srv.slots]
    srv.run(reqs, [0.0] * len(reqs))
    assert [s.held() for s in srv.slots] == held
    for r in reqs:
        assert np.array_equal(bits(r.out), bits(torch.from_numpy(oracle.radix_sort(r.keys.numpy()))))
