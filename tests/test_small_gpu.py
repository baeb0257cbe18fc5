"""GPU parity of the dispatcher's small-array path (Algorithm 5's branch for
arrays below its threshold): one CTA sorts the whole array in shared memory,
in one launch, against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

ALL = [torch.int32, torch.int64, torch.uint32, torch.uint64, torch.float32, torch.float64]


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    evo.table_clear()
    return evo


def bits(t):
    a = t.cpu().numpy()
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def gen(n, dtype, seed):
    from paper_2505_18681_gb300 import inputs
    return inputs.generate("float_mix" if dtype.is_floating_point else "gaussian", n, dtype, seed=seed,
                           device="cuda")


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("cap,sizes", [(0, [2, 3, 1000, 4095, 4096, 4097]), (8192, [8191, 8192, 8193]),
                                       (1024, [1023, 1024, 1025])])
def test_sizes_straddling_the_cut_over(evo, dtype, cap, sizes):
    """Keys and stable pairs, ascending and descending, in and out of place,
    on both sides of the cut-over (the default 4096, and explicit ones)."""
    for n in sizes:
        x = gen(n, dtype, seed=n)
        v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
        xk = x.cpu().numpy()
        ek, ev = oracle.radix_sort(xk, v.cpu().numpy())
        y = torch.empty_like(x)
        evo.sort(x, out=y, small_cap=cap)
        yk, yv = torch.empty_like(x), torch.empty_like(v)
        evo.sort_pairs(x, v, yk, yv, small_cap=cap)
        z = x.clone()
        evo.sort(z, small_cap=cap)
        d = torch.empty_like(x)
        evo.sort(x, out=d, small_cap=cap, descending=True)
        evo.sync()
        ebits = ek.view(bits(y).dtype)
        assert np.array_equal(bits(y), ebits) and np.array_equal(bits(z), ebits), (n, cap)
        assert np.array_equal(bits(yk), ebits) and np.array_equal(yv.cpu().numpy(), ev), (n, cap)
        # descending: the stable descending order is the reverse of the
        # ascending order of the complemented keys; keys-only it is the
        # ascending result reversed
        assert np.array_equal(bits(d), ebits[::-1]), (n, cap)


def test_one_launch_for_a_thousand_keys(evo):
    """A 1,000-key sort with the choice left to the dispatcher is one kernel
    launch (no histogram, scan, passes or scratch allocation)."""
    x = gen(1000, torch.int32, seed=1)
    y = torch.empty_like(x)
    evo.sort(x, out=y)
    evo.sync()
    k0 = evo.kernel_launches()
    evo.profile(True)
    try:
        evo.sort(x, out=y)
        evo.sync()
        recs = evo.profile_read()
    finally:
        evo.profile(False)
    assert evo.kernel_launches() - k0 == 1
    assert [r["kind"] for r in recs] == ["small"]
    assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))


def test_explicit_algorithm_bypasses_the_small_path(evo):
    """algo='radix' keeps the radix sort at any size unless small_cap is
    given; small_cap=1 turns the path off for AUTO too."""
    x = gen(1000, torch.int64, seed=2)
    y = torch.empty_like(x)
    for kw in ({"algo": "radix"}, {"small_cap": 1}):
        k0 = evo.kernel_launches()
        evo.sort(x, out=y, **kw)
        evo.sync()
        assert evo.kernel_launches() - k0 > 1, kw
        assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))
    k0 = evo.kernel_launches()
    evo.sort(x, out=y, algo="radix", small_cap=2048)
    evo.sync()
    assert evo.kernel_launches() - k0 == 1


def test_single_key_needs_no_launch(evo):
    x = gen(1, torch.int64, seed=3)
    y = torch.empty_like(x)
    k0 = evo.kernel_launches()
    evo.sort(x, out=y)
    evo.sort(x)
    evo.sync()
    assert evo.kernel_launches() == k0 and torch.equal(x, y)


def test_bad_cut_over_rejected(evo):
    x = gen(100, torch.int32, seed=4)
    with pytest.raises(evo.EvoSortError) as ei:
        evo.sort(x, small_cap=9000)
    assert ei.value.status == "ERR_INVALID"
