"""GPU parity of the dispatcher's ordered path against the oracle.

With a tuned table loaded and AUTO parameters, an input whose sample is in
order (or in reverse order, keys only) is copied (reversed) with every key
checked against its successor; one key out of order sends the sort to the
radix path.  Either way the output is the oracle's, bit for bit, and key /
value sorts stay stable."""
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


def bits(a):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def records(evo, fn):
    evo.sync()
    evo.profile(True)
    fn()
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync()
    return [(r["kind"], r["pass"]) for r in recs]


def sorted_input(evo, n, dtype, seed):
    """A sorted array with duplicates (the library's radix sort of seeded
    keys; the expected output is the oracle's all the same)."""
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("float_mix" if dtype.is_floating_point else "uniform1000" if n % 2 else "uniform",
                        n, dtype, seed=seed, device="cuda")
    y = torch.empty_like(x)
    evo.sort(x, out=y, algo="radix")
    evo.sync()
    return y


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float32, torch.float64], ids=str)
@pytest.mark.parametrize("n", [70_001, 3_000_017])
def test_sorted_input_is_a_checked_copy(evo, dtype, n):
    x = sorted_input(evo, n, dtype, seed=n)
    y = torch.empty_like(x)
    rec = records(evo, lambda: evo.sort(x, out=y))
    assert ("ordered", 0) in rec and not any(k == "radix_onesweep" for k, _ in rec)
    assert np.array_equal(bits(y), bits(oracle.radix_sort(x.cpu().numpy())))


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float64], ids=str)
def test_reversed_input_is_a_reversed_copy(evo, dtype):
    n = 2_000_003
    x = sorted_input(evo, n, dtype, seed=4).flip(0).contiguous()
    y = torch.empty_like(x)
    rec = records(evo, lambda: evo.sort(x, out=y))
    assert ("ordered", 2) in rec and not any(k == "radix_onesweep" for k, _ in rec)
    assert np.array_equal(bits(y), bits(oracle.radix_sort(x.cpu().numpy())))


def test_in_place_equal_and_descending(evo):
    n = 1_000_003
    x = sorted_input(evo, n, torch.int64, seed=8)
    want = bits(oracle.radix_sort(x.cpu().numpy()))
    z = x.clone()
    rec = records(evo, lambda: evo.sort(z))
    assert ("ordered", 1) in rec
    assert np.array_equal(bits(z), want)
    e = torch.full((n,), -77, dtype=torch.int32, device="cuda")
    f = torch.empty_like(e)
    evo.sort(e, out=f)
    evo.sync()
    assert torch.equal(e, f)
    d = x.flip(0).contiguous()   # descending input, descending sort: a copy
    g = torch.empty_like(d)
    rec = records(evo, lambda: evo.sort(d, out=g, descending=True))
    assert ("ordered", 0) in rec
    assert np.array_equal(bits(g), want[::-1])


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_one_key_out_of_order_falls_back_to_radix(evo, dtype):
    n = 4_000_037
    x = sorted_input(evo, n, dtype, seed=9)
    x[1], x[2] = x[2].clone(), x[1].clone()   # stride n // 4096: positions 1 and 2 are not sampled
    x[n - 2] = x[0] - 1 if x[0] > torch.iinfo(dtype).min else x[0]
    y = torch.empty_like(x)
    rec = records(evo, lambda: evo.sort(x, out=y))
    assert ("ordered", 0) in rec and any(k == "radix_onesweep" for k, _ in rec) or \
        not any(k == "ordered" for k, _ in rec)
    assert np.array_equal(bits(y), bits(oracle.radix_sort(x.cpu().numpy())))


def test_pairs_in_order_and_reversed(evo):
    n = 1_500_007
    x = sorted_input(evo, n, torch.int64, seed=11)
    v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
    ko, vo = torch.empty_like(x), torch.empty_like(v)
    rec = records(evo, lambda: evo.sort_pairs(x, v, ko, vo))
    assert ("ordered", 0) in rec
    wk, wv = oracle.radix_sort(x.cpu().numpy(), np.arange(n, dtype=np.uint32))
    assert np.array_equal(ko.cpu().numpy(), wk)
    assert np.array_equal(vo.cpu().view(torch.int32).numpy().view(np.uint32), wv)
    r = x.flip(0).contiguous()   # reversed with equal keys: not a reversal, radix keeps them stable
    rec = records(evo, lambda: evo.sort_pairs(r, v, ko, vo))
    assert not any(k == "ordered" for k, _ in rec)
    wk, wv = oracle.radix_sort(r.cpu().numpy(), np.arange(n, dtype=np.uint32))
    assert np.array_equal(ko.cpu().numpy(), wk)
    assert np.array_equal(vo.cpu().view(torch.int32).numpy().view(np.uint32), wv)
