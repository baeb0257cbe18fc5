"""GPU parity of descending sorts against the oracle.

Keys only: the descending result is the oracle's ascending result reversed
(equal keys are identical bit patterns).  Pairs: the stable descending sort
keeps equal keys' values in input order; its expected value is the oracle's
stable ascending sort of the complemented order (integers: the bitwise
complement reverses the order; floats: the complement of the oracle's
total-order bits), with the keys gathered by the resulting permutation."""
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


def bits(a):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def gen(dist, n, dtype, seed=42):
    from paper_2505_18681_gb300 import inputs
    if dtype.is_floating_point:
        dist = "float_mix"
    return inputs.generate(dist, n, dtype, seed=seed, device="cuda")


def expected_desc_perm(x: np.ndarray) -> np.ndarray:
    """Stable descending order of x by the total order, from the oracle."""
    idx = np.arange(x.size, dtype=np.uint32)
    if x.dtype.kind in "iu":
        _, perm = oracle.radix_sort(~x, idx)
        return perm
    t = np.array([oracle.ordered_bits(int(u), x.dtype) for u in bits(x)], dtype=np.uint64)
    _, perm = oracle.radix_sort(~t, idx)
    return perm


ALL = [torch.int32, torch.int64, torch.uint32, torch.uint64, torch.float32, torch.float64]


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("n", [1, 2, 33, 4097, 100_003, 3_000_017])
def test_keys_descending_radix(evo, dtype, n):
    x = gen("gaussian" if n > 1000 else "uniform", n, dtype)
    want = oracle.radix_sort(x.cpu().numpy())[::-1]
    y = torch.empty_like(x)
    evo.sort(x, out=y, algo="radix", descending=True)
    evo.sync()
    assert np.array_equal(bits(y), bits(np.ascontiguousarray(want)))


@pytest.mark.parametrize("dtype", [torch.int32, torch.float64], ids=str)
def test_keys_descending_merge(evo, dtype):
    x = gen("uniform", 200_003, dtype)
    want = oracle.radix_sort(x.cpu().numpy())[::-1]
    y = torch.empty_like(x)
    evo.sort(x, out=y, algo="merge", descending=True)
    evo.sync()
    assert np.array_equal(bits(y), bits(np.ascontiguousarray(want)))


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("algo", ["radix", "merge"])
def test_pairs_descending_stable(evo, dtype, algo):
    n = 20_011
    x = gen("distinct16", n, dtype)          # many equal keys: stability shows
    v = torch.arange(n, dtype=torch.int32, device="cuda").view(torch.uint32)
    perm = expected_desc_perm(x.cpu().numpy())
    ko, vo = torch.empty_like(x), torch.empty_like(v)
    evo.sort_pairs(x, v, ko, vo, algo=algo, descending=True)
    evo.sync()
    assert np.array_equal(vo.cpu().numpy(), perm)
    assert np.array_equal(bits(ko), bits(x.cpu().numpy()[perm]))


def test_segmented_descending(evo):
    from paper_2505_18681_gb300 import inputs
    lens = torch.tensor([0, 1, 31, 300, 5000, 20_000, 70_001], dtype=torch.int64)
    keys, offs = inputs.segmented_keys(lens, torch.int32, seed=5, device="cuda")
    asc = oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))
    want = asc.copy()
    o = offs.tolist()
    for a, b in zip(o[:-1], o[1:]):
        want[a:b] = asc[a:b][::-1]
    evo.segmented_sort(keys, offs.to("cuda"), descending=True)
    evo.sync()
    assert np.array_equal(keys.cpu().numpy(), want)


def test_descending_through_the_dispatcher_and_host_batch(evo):
    """With a tuned table the class is read in the sort's direction; the
    result is the descending sort either way, on device and host arrays."""
    evo.table_clear()
    evo.table_load(os.path.join(ROOT, "paper_2505_18681_gb300", "tuned", "gb300_int64.txt"))
    try:
        for dist in ("sorted", "reverse", "distinct16"):
            x = gen(dist, 3_000_017, torch.int64)
            want = np.ascontiguousarray(oracle.radix_sort(x.cpu().numpy())[::-1])
            y = torch.empty_like(x)
            evo.sort(x, out=y, descending=True)
            evo.sync()
            assert np.array_equal(y.cpu().numpy(), want), dist
            h = x.cpu().pin_memory()
            out = torch.empty_like(h).pin_memory()
            evo.sort_host_batch([h], [out], descending=True)
            evo.sync()
            assert np.array_equal(out.numpy(), want), dist
    finally:
        evo.table_clear()
