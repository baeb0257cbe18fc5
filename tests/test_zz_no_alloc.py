"""The sort entry point that allocates no memory, called through the C ABI.

Callers such as plugins inside another framework's execute path, which owns
all device memory, cannot let a library allocate; evosort_sort_noalloc sorts
with a fixed scratch buffer inside the library instead.  Its results are
checked against the CPU oracle and against the allocating entry point, on two
calls in a row (the calls share the buffer), and at the edge of the buffer's
capacity for both key widths.  This file is named so that pytest collects it
last: if it fails, a run that stops at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

CODES = {torch.int32: 0, torch.int64: 1, torch.float64: 5}
BUFFER = 64 << 20


@pytest.fixture(scope="module")
def lib():
    import paper_2505_18681_gb300 as evo
    lib = evo.library()
    lib.evosort_sort_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                         ctypes.c_void_p]
    lib.evosort_sort_noalloc.restype = ctypes.c_int
    return lib


def _allocating(x):
    """The existing allocating entry point's result."""
    import paper_2505_18681_gb300 as evo
    y = torch.empty_like(x)
    evo.sort(x, out=y)
    evo.sync()
    return y


def _oracle(x):
    a = oracle.radix_sort(x.cpu().numpy())
    return torch.from_numpy(a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64))


def _bits(t):
    return t.cpu().view(torch.int32 if t.element_size() == 4 else torch.int64)


def _largest_accepted(dtype):
    """Largest n whose default-plan scratch fits the fixed buffer."""
    import paper_2505_18681_gb300 as evo
    lo, hi = 1, 1 << 26
    while lo < hi:
        m = (lo + hi + 1) // 2
        if evo.workspace_bytes(m, dtype, algo="radix") <= BUFFER:
            lo = m
        else:
            hi = m - 1
    return lo


def test_matches_oracle_and_allocating_sort_on_two_calls_in_a_row(lib):
    from paper_2505_18681_gb300 import inputs
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(torch.int64, "gaussian", 3_000_017), (torch.int32, "uniform", 5_000_011),
             (torch.float64, "float_mix", 1_000_003)]
    for dtype, dist, n in cases:
        for seed in (1, 2):   # two calls in a row share the fixed scratch buffer
            x = inputs.generate(dist, n, dtype, seed=seed, device="cuda")
            out = torch.empty_like(x)
            rc = lib.evosort_sort_noalloc(x.data_ptr(), out.data_ptr(), n, CODES[dtype], stream)
            assert rc == 0, lib.evosort_last_error()
            torch.cuda.synchronize()
            assert torch.equal(_bits(out), _bits(_oracle(x))), (dtype, dist, seed)
            assert torch.equal(out.view(torch.uint8), _allocating(x).view(torch.uint8)), (dtype, dist, seed)
    # in place
    x = inputs.generate("zipf", 2_000_003, torch.int64, seed=3, device="cuda")
    expect = _oracle(x)
    assert lib.evosort_sort_noalloc(x.data_ptr(), x.data_ptr(), x.numel(), 1, stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(_bits(x), _bits(expect))


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_capacity_edge(lib, dtype):
    """The largest size whose scratch fits is sorted correctly; one key more
    is rejected before anything runs."""
    from paper_2505_18681_gb300 import inputs
    n = _largest_accepted(dtype)
    x = inputs.generate("uniform", n + 1, dtype, seed=4, device="cuda")
    head = x[:n]
    out = torch.empty_like(head)
    rc = lib.evosort_sort_noalloc(head.data_ptr(), out.data_ptr(), n, CODES[dtype], None)
    assert rc == 0, lib.evosort_last_error()
    torch.cuda.synchronize()
    assert torch.equal(_bits(out), _bits(_oracle(head)))
    big = torch.empty_like(x)
    rc = lib.evosort_sort_noalloc(x.data_ptr(), big.data_ptr(), n + 1, CODES[dtype], None)
    assert rc == 1
    assert b"64 MiB" in lib.evosort_last_error()
