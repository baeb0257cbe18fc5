"""GPU parity of the host-memory batch sort (upload, sort, download pipelined
over three device slots) against the CPU oracle, bit for bit, for every key
type, in place and out of place, pinned and pageable, more arrays than
slots, empty arrays, and with the dispatcher's tuned parameters."""
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIZES = [1000, 0, 100_003, 1, 2_000_001, 5, 777_777]


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


def bits(a):
    a = a.numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def host_arrays(dtype, sizes, pin, dists=("uniform", "gaussian", "sorted", "distinct16", "reverse")):
    from paper_2505_18681_gb300 import inputs
    xs = []
    for i, n in enumerate(sizes):
        dist = "float_mix" if dtype.is_floating_point else dists[i % len(dists)]
        x = inputs.generate(dist, max(n, 1), dtype, seed=100 + i, device="cuda")[:n].cpu().contiguous()
        xs.append(x.pin_memory() if pin and n else x)
    return xs


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.uint32, torch.uint64, torch.float32,
                                   torch.float64], ids=str)
def test_out_of_place_pinned(evo, dtype):
    xs = host_arrays(dtype, SIZES, pin=True)
    keep = [x.clone() for x in xs]
    outs = [torch.empty_like(x).pin_memory() if x.numel() else torch.empty_like(x) for x in xs]
    evo.sort_host_batch(xs, outs, algo="radix")
    evo.sync()
    for x, k, y in zip(xs, keep, outs):
        assert np.array_equal(bits(x), bits(k)), "input changed"
        assert np.array_equal(bits(y), bits(oracle.radix_sort(k.numpy())))


@pytest.mark.parametrize("pin", [True, False], ids=["pinned", "pageable"])
def test_in_place(evo, pin):
    xs = host_arrays(torch.int64, SIZES, pin=pin)
    expect = [oracle.radix_sort(x.numpy().copy()) for x in xs]
    evo.sort_host_batch(xs)
    evo.sync()
    for x, e in zip(xs, expect):
        assert np.array_equal(bits(x), bits(e))


def test_merge_path_and_single_array(evo):
    xs = host_arrays(torch.float64, [300_001], pin=True)
    e = oracle.merge_sort(xs[0].numpy().copy())
    evo.sort_host_batch(xs, algo="merge")
    evo.sync()
    assert np.array_equal(bits(xs[0]), bits(e))


def test_dispatcher_plans_from_host_sample(evo):
    """With a tuned table and AUTO parameters every array gets its class's
    parameters; the result is the sort either way."""
    evo.table_clear()
    evo.table_load(os.path.join(ROOT, "paper_2505_18681_gb300", "tuned", "gb300_int64.txt"))
    try:
        xs = host_arrays(torch.int64, [3_000_000, 2_500_000, 1_000_000, 4_000_000], pin=True,
                         dists=("zipf", "uniform1000", "equal", "distinct16"))
        expect = [oracle.radix_sort(x.numpy().copy()) for x in xs]
        evo.sort_host_batch(xs)
        evo.sync()
        for x, e in zip(xs, expect):
            assert np.array_equal(bits(x), bits(e))
    finally:
        evo.table_clear()


def test_ordered_on_the_callers_stream(evo):
    """Work enqueued on the caller's stream after the batch sees its results:
    a device copy of the host output made on that stream holds sorted keys."""
    s = torch.cuda.Stream()
    xs = host_arrays(torch.int32, [1_500_000, 900_000, 1_200_000, 50_000], pin=True)
    outs = [torch.empty_like(x).pin_memory() for x in xs]
    with torch.cuda.stream(s):
        evo.sort_host_batch(xs, outs, algo="radix", stream=s)
        evo.sync(s)
    for x, y in zip(xs, outs):
        assert np.array_equal(bits(y), bits(oracle.radix_sort(x.numpy().copy())))
