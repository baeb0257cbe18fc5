"""The sort entry point that allocates no memory, called through the C ABI.

Callers such as plugins inside another framework's execute path, which owns
all device memory, cannot let a library allocate; evosort_sort_noalloc sorts
with a fixed scratch buffer inside the library instead.  This file is named so
that pytest collects it last: if it fails, a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2505_18681_gb300 as evo
    lib = evo.library()
    lib.evosort_sort_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                         ctypes.c_void_p]
    lib.evosort_sort_noalloc.restype = ctypes.c_int
    return lib


def _reference(x):
    """The existing allocating entry point's result."""
    import paper_2505_18681_gb300 as evo
    y = torch.empty_like(x)
    evo.sort(x, out=y)
    evo.sync()
    return y


def test_matches_allocating_sort_on_two_calls_in_a_row(lib):
    from paper_2505_18681_gb300 import inputs
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(torch.int64, "gaussian", 3_000_017), (torch.int32, "uniform", 5_000_011),
             (torch.float64, "float_mix", 1_000_003)]
    for dtype, dist, n in cases:
        code = {torch.int32: 0, torch.int64: 1, torch.float64: 5}[dtype]
        for seed in (1, 2):   # two calls in a row share the fixed scratch buffer
            x = inputs.generate(dist, n, dtype, seed=seed, device="cuda")
            ref = _reference(x)
            out = torch.empty_like(x)
            rc = lib.evosort_sort_noalloc(x.data_ptr(), out.data_ptr(), n, code, stream)
            assert rc == 0, lib.evosort_last_error()
            torch.cuda.synchronize()
            assert torch.equal(out.view(torch.uint8), ref.view(torch.uint8)), (dtype, dist, seed)
    # in place
    x = inputs.generate("zipf", 2_000_003, torch.int64, seed=3, device="cuda")
    ref = _reference(x)
    assert lib.evosort_sort_noalloc(x.data_ptr(), x.data_ptr(), x.numel(), 1, stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(x, ref)


def test_rejects_sizes_beyond_its_buffer(lib):
    n = 20_000_000   # 160 MB of int64 keys: more scratch than the fixed 64 MiB
    x = torch.empty(n, dtype=torch.int64, device="cuda")
    rc = lib.evosort_sort_noalloc(x.data_ptr(), x.data_ptr(), n, 1, None)
    assert rc == 1
    assert b"64 MiB" in lib.evosort_last_error()
