"""GPU parity of range-reduced radix sorts against the oracle.

When the mapped keys span fewer 8-bit digits than the raw digits that vary
(keys of both signs near zero differ in every high byte), the passes rank
key - min instead of the key.  The result must be the oracle's sort bit for
bit, stable for pairs, in every direction and kernel; the profile records
show how many passes ran."""
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


def active_passes(evo, fn):
    """Runs fn under profiling; the number of onesweep passes that ran."""
    evo.sync()
    evo.profile(True)
    fn()
    recs = evo.profile_read()
    evo.profile(False)
    evo.sync()
    return len({r["pass"] for r in recs if r["kind"] == "radix_onesweep" and r["active"]})


def near_zero(n, dtype, spread, seed):
    """Keys of both signs in [-spread, spread) (uniform, seeded)."""
    g = torch.Generator().manual_seed(seed)
    x = torch.randint(-spread, spread, (n,), generator=g, dtype=torch.int64)
    return x.to(dtype).to("cuda")


@pytest.mark.parametrize("dtype,spread,passes", [(torch.int64, 1 << 20, 3), (torch.int64, 1 << 23, 3),
                                                 (torch.int64, 1 << 30, 4), (torch.int32, 1 << 20, 3),
                                                 (torch.int32, 1 << 14, 2)], ids=str)
@pytest.mark.parametrize("n", [5_000, 100_003, 3_000_017])
def test_signed_keys_near_zero(evo, dtype, spread, passes, n):
    x = near_zero(n, dtype, spread, seed=n + spread)
    y = torch.empty_like(x)
    ran = active_passes(evo, lambda: evo.sort(x, out=y, algo="radix"))
    assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))
    assert ran == passes


@pytest.mark.parametrize("width,passes", [((1 << 24) - 1, 3), (1 << 24, 4)])
def test_span_at_a_byte_boundary(evo, width, passes):
    """max - min = 2^24 - 1 needs three digits, 2^24 needs four."""
    n = 1_000_003
    lo = -(1 << 23) - 12345
    g = torch.Generator().manual_seed(width)
    x = torch.randint(lo, lo + width + 1, (n,), generator=g, dtype=torch.int64)
    x[7] = lo
    x[n - 3] = lo + width
    x = x.cuda()
    y = torch.empty_like(x)
    ran = active_passes(evo, lambda: evo.sort(x, out=y, algo="radix"))
    assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))
    assert ran == passes


def test_unsigned_keys_straddling_a_byte_boundary(evo):
    """[2^32 - 2^14, 2^32 + 2^14): five raw digits vary, the span needs two
    (wide enough not to be a narrow range for the counting sort)."""
    n = 2_000_011
    g = torch.Generator().manual_seed(5)
    x = (torch.randint(-(1 << 14), 1 << 14, (n,), generator=g, dtype=torch.int64) + (1 << 32))
    x = x.cuda().view(torch.uint64)
    y = torch.empty_like(x)
    ran = active_passes(evo, lambda: evo.sort(x, out=y, algo="radix"))
    want = oracle.radix_sort(x.cpu().view(torch.int64).numpy().view(np.uint64))
    assert np.array_equal(y.cpu().view(torch.int64).numpy().view(np.uint64), want)
    assert ran == 2


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
@pytest.mark.parametrize("pass_kernel", [1, 2])
def test_pairs_stable_and_both_kernels(evo, dtype, pass_kernel):
    """Many equal keys (spread 300): values keep input order among them."""
    n = 1_500_007
    x = near_zero(n, dtype, 300, seed=11)
    v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
    ko, vo = torch.empty_like(x), torch.empty_like(v)
    ran = active_passes(evo, lambda: evo.sort_pairs(x, v, ko, vo, algo="radix", pass_kernel=pass_kernel,
                                                    digit_bits=8))
    wk, wv = oracle.radix_sort(x.cpu().numpy(), np.arange(n, dtype=np.uint32))
    assert np.array_equal(ko.cpu().numpy(), wk)
    assert np.array_equal(vo.cpu().view(torch.int32).numpy().view(np.uint32), wv)
    assert ran == 2


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_descending_and_in_place(evo, dtype):
    n = 2_000_003
    x = near_zero(n, dtype, 1 << 19, seed=3)
    want = oracle.radix_sort(x.cpu().numpy())
    y = torch.empty_like(x)
    evo.sort(x, out=y, algo="radix", descending=True)
    evo.sync()
    assert np.array_equal(y.cpu().numpy(), want[::-1])
    z = x.clone()   # in place: three passes, an odd count, end with a copy
    ran = active_passes(evo, lambda: evo.sort(z, algo="radix"))
    assert np.array_equal(z.cpu().numpy(), want)
    assert ran == 3


def test_floats_and_wide_keys_are_not_rebased(evo):
    """Float keys of both signs span the whole mapped range, uniform keys
    need every digit: both sort exactly as before, with every pass."""
    from paper_2505_18681_gb300 import inputs
    for dist, dtype, passes in (("float_mix", torch.float64, 8), ("uniform", torch.int64, 8),
                                ("uniform", torch.int32, 4)):
        x = inputs.generate(dist, 1_000_003, dtype, seed=9, device="cuda")
        y = torch.empty_like(x)
        ran = active_passes(evo, lambda: evo.sort(x, out=y, algo="radix"))
        got = y.cpu().numpy()
        want = oracle.radix_sort(x.cpu().numpy())
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
        assert ran == passes


def test_gaussian_input_runs_three_passes(evo):
    """The bench's Gaussian workload shape (N(0, 1e6), int64): three passes."""
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("gaussian", 4_000_037, torch.int64, seed=42, device="cuda")
    y = torch.empty_like(x)
    ran = active_passes(evo, lambda: evo.sort(x, out=y))
    assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))
    assert ran == 3
