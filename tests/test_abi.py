"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/*.h, and rejects bad arguments before it
touches the device."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_18681_gb300 import _build
    _build.build()
    import paper_2505_18681_gb300 as evo
    return evo.library()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(evosort_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("evosort_sort", "evosort_sort_pairs", "evosort_sync", "evosort_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2505_18681_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(evosort_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    for n in declared_symbols():
        assert hasattr(lib, n)


def test_library_is_built_for_sm103a():
    from paper_2505_18681_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.NVCC_FLAGS)


def _params(lib, **kw):
    import paper_2505_18681_gb300 as evo
    p = evo.Params()
    lib.evosort_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


FAKE = 0x10000   # never dereferenced: every case below fails its host check first


def test_rejects_bad_arguments_without_a_gpu(lib):
    p = _params(lib)
    bp = ctypes.byref(p)
    assert lib.evosort_sort(None, 10, 0, bp) == 1                 # null keys
    assert lib.evosort_sort(FAKE, 10, 9, bp) == 1                 # bad dtype
    assert lib.evosort_sort(FAKE + 2, 10, 0, bp) == 1             # misaligned int32
    assert lib.evosort_sort(FAKE + 4, 10, 1, bp) == 1             # misaligned int64
    assert lib.evosort_sort_to(FAKE, FAKE + 8, 10, 0, bp) == 1    # overlapping in/out
    assert lib.evosort_sort_pairs(FAKE, None, 10, 0, bp) == 1     # null values
    assert lib.evosort_sort_pairs_to(FAKE, FAKE + 4096, FAKE + 8192, FAKE + 4096, 10, 0, bp) == 1
    msg = lib.evosort_last_error()
    assert msg and len(msg) > 0
    # n == 0 is a no-op that never touches the device
    assert lib.evosort_sort(None, 0, 0, bp) == 0
    assert lib.evosort_sort(FAKE, 0, 0, bp) == 0


def test_host_batch_rejects_bad_arguments_without_a_gpu(lib):
    p = _params(lib)
    bp = ctypes.byref(p)
    VP = ctypes.c_void_p * 2
    NS = ctypes.c_size_t * 2
    ins, outs, ns = VP(FAKE, FAKE + 4096), VP(FAKE + 8192, FAKE + 16384), NS(10, 10)
    f = lib.evosort_sort_host_batch
    assert f(ins, outs, ns, 2, 9, bp) == 1                             # bad dtype
    assert f(None, outs, ns, 2, 0, bp) == 1                            # null list
    assert f(ins, VP(FAKE + 8, FAKE + 16384), ns, 2, 0, bp) == 1       # overlapping in/out
    assert f(VP(FAKE + 2, FAKE + 4096), outs, ns, 2, 0, bp) == 1       # misaligned int32
    assert f(VP(None, FAKE + 4096), outs, ns, 2, 0, bp) == 1           # null keys
    bad = _params(lib, digit_bits=3)
    assert f(ins, outs, ns, 2, 0, ctypes.byref(bad)) == 1              # bad parameters
    assert b"host_batch" in lib.evosort_last_error()
    # nothing to sort: no device work at all
    assert f(ins, outs, ns, 0, 0, bp) == 0
    assert f(VP(None, None), VP(None, None), NS(0, 0), 2, 0, bp) == 0


@pytest.mark.parametrize("field,value", [("digit_bits", 3), ("digit_bits", 12), ("algo", 7),
                                         ("rank_mode", 5), ("rank_mode", -1), ("insertion_threshold", 1),
                                         ("insertion_threshold", 4096), ("block_size", 100)])
def test_rejects_bad_params(lib, field, value):
    p = _params(lib, **{field: value})
    assert lib.evosort_sort(FAKE, 10, 0, ctypes.byref(p)) == 1
    assert lib.evosort_workspace_bytes(1000, 0, 0, ctypes.byref(p)) == 0


def test_adaptive_ranking_needs_8_bit_digits(lib):
    for d in (4, 6, 7, 9, 11):
        p = _params(lib, rank_mode=4, digit_bits=d)
        assert lib.evosort_sort(FAKE, 10, 0, ctypes.byref(p)) == 1
    assert b"rank_mode" in lib.evosort_last_error()


def test_workspace_bytes_grows_with_n(lib):
    p = _params(lib)
    a = lib.evosort_workspace_bytes(1000, 0, 0, ctypes.byref(p))
    b = lib.evosort_workspace_bytes(1_000_000, 0, 0, ctypes.byref(p))
    c = lib.evosort_workspace_bytes(1_000_000, 0, 1, ctypes.byref(p))
    assert 0 < a < b < c
    assert b >= 4 * 1_000_000    # at least the ping-pong key buffer


def test_python_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2505_18681_gb300 as evo
    from paper_2505_18681_gb300 import _build
    monkeypatch.setattr(evo, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        evo.library()


def _largest_noalloc(lib, dt):
    """Largest n whose default radix scratch fits 64 MiB (host arithmetic)."""
    import paper_2505_18681_gb300 as evo
    p = evo.make_params(algo="radix")
    lo, hi = 1, 1 << 26
    while lo < hi:
        m = (lo + hi + 1) // 2
        if lib.evosort_workspace_bytes(m, dt, 0, ctypes.byref(p)) <= 64 << 20:
            lo = m
        else:
            hi = m - 1
    return lo


def test_noalloc_limit_matches_its_declaration(lib):
    """The sizes the header quotes for the fixed 64 MiB buffer are the ones
    the workspace arithmetic gives, and one key more is rejected on the host
    (the pointers are never used: the size check comes first)."""
    f = lib.evosort_sort_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    text = re.sub(r"\n\s*\*\s?", " ", open(os.path.join(ROOT, "include", "evosort.h")).read())
    m = re.search(r"about\s+([\d.]+) million 64-bit or ([\d.]+) million 32-bit keys", text)
    assert m, "the limit is quoted in the declaration"
    for dt, quoted, w in ((1, float(m.group(1)), 8), (0, float(m.group(2)), 4)):
        n = _largest_noalloc(lib, dt)
        assert round(n / 1e6, 1) == quoted, (dt, n)
        big = n + 1
        assert f(FAKE, FAKE + big * w + 4096, big, dt, None) == 1
        assert b"64 MiB" in lib.evosort_last_error()
    assert f(FAKE, FAKE, 0, 1, None) == 0              # nothing to sort
    assert f(FAKE, FAKE + 8, 10, 1, None) == 1         # overlapping
    assert f(FAKE + 4, FAKE + 4096, 10, 1, None) == 1  # misaligned
    assert f(FAKE, FAKE + 4096, 10, 9, None) == 1      # bad dtype


def test_shard_entry_points_reject_bad_arguments(lib):
    kr, rh = lib.evosort_key_range, lib.evosort_range_histogram
    assert kr(None, 10, 1, 0, FAKE, None) == 1                       # null keys
    assert kr(FAKE, 10, 9, 0, FAKE, None) == 1                       # bad dtype
    assert kr(FAKE, 10, 1, 0, None, None) == 1                       # null range
    for nbins, shift, dt in ((0, 0, 1), (8193, 0, 1), (16, 64, 1), (16, 32, 0), (16, -1, 1)):
        assert rh(FAKE, 10, dt, 0, 0, shift, nbins, FAKE, None) == 1
    assert rh(FAKE, 10, 1, 0, 0, 0, 16, None, None) == 1              # null counts
    assert b"evosort_range_histogram: bad argument" in lib.evosort_last_error()
    assert rh(None, 0, 1, 0, 0, 0, 16, FAKE, None) == 0               # nothing to count


def test_every_declaration_cites_its_passage():
    """Each entry point's comment (its own or its section's) names the part
    of the paper it follows (an algorithm or section) or says the paper has
    no counterpart."""
    text = open(os.path.join(ROOT, "include", "evosort.h")).read()
    cite = re.compile(r"Algorithm|Section|paper")
    missing = []
    decl = r"^(?:evosort_status|void|size_t|int|uint64_t|const char\*)\s+(evosort_\w+)\s*\("
    for m in re.finditer(decl, text, re.M):
        before = text[:m.start()]
        end = before.rfind("*/")
        own = before[before.rfind("/*", 0, end):end] if end != -1 else ""
        sec_at = before.rfind("/* ----")
        section = text[sec_at:text.find("*/", sec_at)] if sec_at != -1 else ""
        if not (cite.search(own) or cite.search(section)):
            missing.append(m.group(1))
    assert not missing, missing
    assert len(declared_symbols()) >= 30


def test_resolve_reports_when_the_small_path_applies():
    """evosort_resolve reports small_cap as the sort applies it: the default
    cut-over when the algorithm is left to the dispatcher, off (1) for an
    explicit algorithm unless a cut-over is given."""
    import torch
    import paper_2505_18681_gb300 as evo
    assert evo.resolve(1000, torch.int32)["small_cap"] == 4096
    assert evo.resolve(1000, torch.int32, algo="auto")["small_cap"] == 4096
    assert evo.resolve(1000, torch.int32, algo="radix")["small_cap"] == 1
    assert evo.resolve(1000, torch.int64, algo="merge")["small_cap"] == 1
    assert evo.resolve(1000, torch.int32, algo="radix", small_cap=2048)["small_cap"] == 2048
    assert evo.resolve(1000, torch.int32, algo="auto", small_cap=1)["small_cap"] == 1


class _FakeTensor:
    """Stands in for a CUDA tensor in the binding's argument check."""

    def __init__(self, index, contiguous=True, cuda=True):
        import torch
        self.device = torch.device("cuda", index)
        self.is_cuda = cuda
        self._contiguous = contiguous

    def is_contiguous(self):
        return self._contiguous


def test_binding_wants_tensors_on_the_current_device(monkeypatch):
    import torch
    import paper_2505_18681_gb300 as evo
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 1)
    evo._need_cuda(_FakeTensor(1), None, _FakeTensor(1))
    with pytest.raises(ValueError, match="one device"):
        evo._need_cuda(_FakeTensor(1), _FakeTensor(0))
    with pytest.raises(ValueError, match="current device"):
        evo._need_cuda(_FakeTensor(0))
    with pytest.raises(ValueError, match="contiguous"):
        evo._need_cuda(_FakeTensor(1, contiguous=False))
    with pytest.raises(ValueError, match="CUDA device"):
        evo._need_cuda(_FakeTensor(1, cuda=False))
    evo._need_cuda(None)
