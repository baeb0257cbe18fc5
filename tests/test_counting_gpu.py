"""GPU parity of the radix path's narrow-range counting sort against the
oracle.

When the keys span between 256 and 8191 values (keys only, 8-bit digits),
the radix sort counts every key by value and writes the output from the
counts; no pass runs.  Outside that window (or for key / value sorts, or
inputs already in order) the passes run as before."""
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


def bits(a):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def passes_run(evo, fn):
    """(onesweep passes that ran, whether the fixup copied)."""
    evo.sync()
    evo.profile(True)
    fn()
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync()
    ran = len({r["pass"] for r in recs if r["kind"] == "radix_onesweep" and r["active"]})
    fix = any(r["kind"] == "radix_fixup" and r["active"] for r in recs)
    return ran, fix


def narrow(n, dtype, lo, span, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.randint(lo, lo + span, (n,), generator=g, dtype=torch.int64)
    x[n // 3] = lo
    x[n // 2] = lo + span - 1   # the span is exactly `span` values
    return x.to(dtype).cuda()


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
@pytest.mark.parametrize("width,counted", [(255, False), (256, True), (998, True), (8191, True), (8192, False)])
@pytest.mark.parametrize("n", [5_003, 3_000_017])
def test_width_window(evo, dtype, width, counted, n):
    """max - min = width: counted for 256 <= width < 8192, passes otherwise."""
    x = narrow(n, dtype, -117, width + 1, seed=width + n)
    y = torch.empty_like(x)
    ran, fix = passes_run(evo, lambda: evo.sort(x, out=y, algo="radix"))
    assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))
    if counted:
        assert ran == 0 and not fix
    else:
        assert ran >= 1


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_descending_in_place_and_floats(evo, dtype):
    n = 2_000_003
    x = narrow(n, dtype, 5000, 3000, seed=1)
    want = oracle.radix_sort(x.cpu().numpy())
    y = torch.empty_like(x)
    evo.sort(x, out=y, algo="radix", descending=True)
    evo.sync()
    assert np.array_equal(y.cpu().numpy(), want[::-1])
    z = x.clone()
    ran, fix = passes_run(evo, lambda: evo.sort(z, algo="radix"))
    assert ran == 0 and not fix
    assert np.array_equal(z.cpu().numpy(), want)
    # adjacent float32 bit patterns: a narrow range in the float order
    g = torch.Generator().manual_seed(2)
    b = (torch.randint(0, 3000, (n,), generator=g, dtype=torch.int64) + 0x3F800000).to(torch.int32)
    f = b.view(torch.float32).cuda()
    h = torch.empty_like(f)
    ran, _ = passes_run(evo, lambda: evo.sort(f, out=h, algo="radix"))
    assert ran == 0
    assert np.array_equal(bits(h), bits(oracle.radix_sort(f.cpu().numpy())))


def test_pairs_and_sorted_input_keep_their_paths(evo):
    n = 1_000_003
    x = narrow(n, torch.int64, 0, 1000, seed=3)
    v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
    ko, vo = torch.empty_like(x), torch.empty_like(v)
    ran, _ = passes_run(evo, lambda: evo.sort_pairs(x, v, ko, vo, algo="radix"))
    assert ran >= 1
    wk, wv = oracle.radix_sort(x.cpu().numpy(), np.arange(n, dtype=np.uint32))
    assert np.array_equal(ko.cpu().numpy(), wk)
    assert np.array_equal(vo.cpu().view(torch.int32).numpy().view(np.uint32), wv)
    s = torch.sort(x).values.contiguous()   # in order: the histogram's copy, not counting
    t = torch.empty_like(s)
    ran, fix = passes_run(evo, lambda: evo.sort(s, out=t, algo="radix"))
    assert ran == 0 and fix
    assert torch.equal(s, t)
