"""GPU parity of the dispatcher's few-values path against the oracle.

With a tuned table loaded and AUTO parameters, an array whose sample holds
at most 64 distinct keys is sorted by counting over those values (keys
only); a key the sample did not see sends the sort back to the radix path.
Either way the output is the oracle's, bit for bit."""
import os

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "paper_2505_18681_gb300", "tuned")


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    evo.table_clear()
    evo.table_load(os.path.join(TABLES, "gb300_int32.txt"))
    evo.table_load(os.path.join(TABLES, "gb300_int64.txt"))
    yield evo
    evo.table_clear()


def few_values(n, dtype, k, seed):
    """n keys, each one of k seeded values (floats: including -0.0, +0.0, a
    NaN and -inf; unsigned keys: the bit patterns of signed ones)."""
    g = torch.Generator().manual_seed(seed)
    if dtype.is_floating_point:
        vals = (torch.rand(k, generator=g, dtype=torch.float64) * 2e6 - 1e6).to(dtype)
        specials = torch.tensor([-0.0, 0.0, float("nan"), float("-inf")], dtype=dtype)
        vals[:min(4, k)] = specials[:min(4, k)]
    elif dtype in (torch.int32, torch.uint32):
        vals = torch.randint(-(1 << 31), 1 << 31, (k,), generator=g, dtype=torch.int64).to(torch.int32)
    else:
        vals = torch.randint(-(1 << 62), 1 << 62, (k,), generator=g, dtype=torch.int64)
    idx = torch.randint(0, k, (n,), generator=g)
    x = vals[idx].cuda()
    if dtype == torch.uint32:
        return x.view(torch.uint32)
    if dtype == torch.uint64:
        return x.view(torch.uint64)
    return x


def expected(x):
    """The oracle's sort of x (numpy array of x's own dtype)."""
    h = x
    if x.dtype == torch.uint32:
        a = h.view(torch.int32).cpu().numpy().view(np.uint32)
    elif x.dtype == torch.uint64:
        a = h.view(torch.int64).cpu().numpy().view(np.uint64)
    else:
        a = h.cpu().numpy()
    return oracle.radix_sort(a)


def bits(a):
    if isinstance(a, torch.Tensor):
        if a.dtype == torch.uint32:
            a = a.view(torch.int32)
        elif a.dtype == torch.uint64:
            a = a.view(torch.int64)
        a = a.cpu().numpy()
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def kinds(evo, fn):
    evo.sync()
    evo.profile(True)
    fn()
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync()
    return [(r["kind"], r["pass"]) for r in recs]


ALL = [torch.int32, torch.int64, torch.uint32, torch.uint64, torch.float32, torch.float64]


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("n", [70_001, 1_000_003, 5_000_011])
def test_few_values_counting_path(evo, dtype, n):
    x = few_values(n, dtype, 16, seed=n)
    y = torch.empty_like(x)
    rec = kinds(evo, lambda: evo.sort(x, out=y))
    assert ("dict", 1) in rec and not any(k == "radix_onesweep" for k, _ in rec)
    assert np.array_equal(bits(y), bits(expected(x)))


@pytest.mark.parametrize("dtype", [torch.int32, torch.float64], ids=str)
def test_descending_and_in_place(evo, dtype):
    n = 2_000_003
    x = few_values(n, dtype, 40, seed=7)
    want = bits(expected(x))
    y = torch.empty_like(x)
    rec = kinds(evo, lambda: evo.sort(x, out=y, descending=True))
    assert ("dict", 1) in rec
    assert np.array_equal(bits(y), want[::-1])
    z = x.clone()
    evo.sort(z)
    evo.sync()
    assert np.array_equal(bits(z), want)


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_value_missed_by_the_sample_falls_back_to_radix(evo, dtype):
    """One key off the sample's stride holds a value no sampled key has: the
    count finds it, the radix path sorts the untouched input."""
    n = 4_000_037
    x = few_values(n, dtype, 16, seed=3)
    x[1] = 12345 if dtype == torch.int32 else -(1 << 40) - 7   # stride n // 4096: index 1 is not sampled
    y = torch.empty_like(x)
    rec = kinds(evo, lambda: evo.sort(x, out=y))
    assert ("dict", 0) in rec and ("dict", 1) not in rec
    assert any(k == "radix_onesweep" for k, _ in rec)
    assert np.array_equal(bits(y), bits(expected(x)))


def test_pairs_and_small_arrays_take_the_other_paths(evo):
    n = 1_000_003
    x = few_values(n, torch.int64, 16, seed=5)
    v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
    ko, vo = torch.empty_like(x), torch.empty_like(v)
    rec = kinds(evo, lambda: evo.sort_pairs(x, v, ko, vo))
    assert not any(k == "dict" for k, _ in rec)
    wk, wv = oracle.radix_sort(x.cpu().numpy(), np.arange(n, dtype=np.uint32))
    assert np.array_equal(ko.cpu().numpy(), wk)
    assert np.array_equal(vo.cpu().view(torch.int32).numpy().view(np.uint32), wv)
    s = few_values(50_000, torch.int64, 16, seed=6)   # below the path's minimum size
    t = torch.empty_like(s)
    rec = kinds(evo, lambda: evo.sort(s, out=t))
    assert not any(k == "dict" for k, _ in rec)
    assert np.array_equal(t.cpu().numpy(), oracle.radix_sort(s.cpu().numpy()))
