"""GPU parity of the mergesort path (Algorithm 3) against the CPU oracle.

The oracle's bottom-up mergesort (O2) with the same insertion threshold is
the reference; since the result is the unique stable sort, it also equals the
oracle's radix sort (checked in the oracle's own tests).
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

ALL = [torch.int32, torch.int64, torch.uint32, torch.uint64, torch.float32, torch.float64]


def bits(t):
    a = t.cpu().numpy()
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def gen(dist, n, dtype, seed=42):
    from paper_2505_18681_gb300 import inputs
    if dtype.is_floating_point and dist != "float_mix":
        dist = "uniform"
    return inputs.generate(dist, n, dtype, seed=seed, device="cuda")


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


def check(evo, x, tins=32, pairs=False, inplace=False):
    host = x.cpu().numpy()
    if pairs:
        v = torch.arange(x.numel(), dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
        ek, ev = oracle.merge_sort(host, v.cpu().numpy(), chunk_size=tins)
        if inplace:
            k, vv = x.clone(), v.clone()
            evo.sort_pairs(k, vv, algo="merge", insertion_threshold=tins)
        else:
            k, vv = torch.empty_like(x), torch.empty_like(v)
            evo.sort_pairs(x, v, k, vv, algo="merge", insertion_threshold=tins)
        evo.sync()
        assert np.array_equal(bits(k), ek.view(bits(k).dtype))
        assert np.array_equal(vv.cpu().numpy(), ev)
    else:
        e = oracle.merge_sort(host, chunk_size=tins)
        if inplace:
            y = x.clone()
            evo.sort(y, algo="merge", insertion_threshold=tins)
        else:
            y = torch.empty_like(x)
            evo.sort(x, out=y, algo="merge", insertion_threshold=tins)
        evo.sync()
        assert np.array_equal(bits(y), e.view(bits(y).dtype))


def test_config_1e6_int32_seed0_tins32(evo):
    """1e6 int32 keys uniform over the full range, seed 0, insertion threshold 32."""
    x = gen("uniform", 1_000_000, torch.int32, seed=0)
    check(evo, x, tins=32)
    check(evo, x, tins=32, inplace=True)


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 4095, 4096, 4097, 3 * 4096 + 17, 100_003])
def test_sizes(evo, dtype, n):
    check(evo, gen("uniform", n, dtype))


@pytest.mark.parametrize("tins", [2, 3, 7, 32, 100, 257, 2048])
def test_insertion_thresholds(evo, tins):
    """Base-run lengths that are not powers of two give tiles that straddle
    merge pairs in the global rounds."""
    for n in (50_001, 300_007):
        check(evo, gen("uniform", n, torch.int64), tins=tins)
        check(evo, gen("distinct16", n, torch.int32), tins=tins, pairs=True)


@pytest.mark.parametrize("dist", ["gaussian", "sorted", "reverse", "nearly_sorted", "distinct16", "zipf",
                                  "equal", "uniform1000"])
def test_distributions(evo, dist):
    x = gen(dist, 200_003, torch.int64)
    check(evo, x)
    check(evo, x, pairs=True, inplace=True)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=str)
def test_float_pairs_stable(evo, dtype):
    x = gen("float_mix", 150_001, dtype)
    check(evo, x, pairs=True)
    check(evo, x, tins=5, pairs=True, inplace=True)


def test_matches_radix(evo):
    """Both algorithms give the same bits (the unique stable sort)."""
    x = gen("zipf", 400_009, torch.int64)
    a, b = torch.empty_like(x), torch.empty_like(x)
    evo.sort(x, out=a, algo="merge", insertion_threshold=64)
    evo.sort(x, out=b, algo="radix")
    evo.sync()
    assert torch.equal(a, b)
