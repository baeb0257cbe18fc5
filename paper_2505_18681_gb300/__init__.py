"""GB300 (sm_103a) sort library: Python binding of the C ABI in include/evosort.h.

This module only marshals arguments: it passes device pointers, sizes, the
current CUDA stream and the parameter struct to ``libevosort.so``; every step
of every sort runs in the library's CUDA kernels.  There is no CPU path: if
the library has not been built, every call raises.

    import torch, paper_2505_18681_gb300 as evo
    x = torch.randint(-2**31, 2**31 - 1, (10**6,), dtype=torch.int32, device="cuda")
    evo.sort(x)                          # in place, LSD radix (Algorithms 4a/4b)
    y = evo.sort(x, out=torch.empty_like(x), algo="merge", insertion_threshold=32)
    k, v = evo.sort_pairs(keys, torch.arange(n, dtype=torch.uint32, device="cuda"))
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

__all__ = ["sort", "sort_pairs", "segmented_sort", "sync", "release", "workspace_bytes", "kernel_launches", "set_wait_limit",
           "profile", "profile_read",
           "EvoSortError", "Params", "library", "DTYPES"]

DTYPES = {torch.int32: 0, torch.int64: 1, torch.uint32: 2, torch.uint64: 3,
          torch.float32: 4, torch.float64: 5}
ALGOS = {"auto": -1, "radix": 0, "merge": 1, None: -1, -1: -1, 0: 0, 1: 1}
STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_NOMEM", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_UNSUPPORTED"}


class EvoSortError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(code, code), message))
        self.code = code
        self.status = STATUS.get(code, str(code))


class Params(ctypes.Structure):
    """Mirror of ``evosort_params``."""
    _fields_ = [("algo", ctypes.c_int), ("digit_bits", ctypes.c_int), ("keys_per_thread", ctypes.c_int),
                ("block_size", ctypes.c_int), ("insertion_threshold", ctypes.c_int),
                ("rank_mode", ctypes.c_int), ("seg_block_cap", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("descending", ctypes.c_int), ("pass_kernel", ctypes.c_int),
                ("adapt_later", ctypes.c_int), ("adapt_first", ctypes.c_int), ("seg_warp_cap", ctypes.c_int),
                ("small_cap", ctypes.c_int), ("seg_giant", ctypes.c_longlong)]


class GAConfig(ctypes.Structure):
    """Mirror of ``evosort_ga_config``."""
    _fields_ = [("population", ctypes.c_int), ("generations", ctypes.c_int), ("crossover_p", ctypes.c_double),
                ("mutation_p", ctypes.c_double), ("gene_mutation_p", ctypes.c_double), ("elite", ctypes.c_int),
                ("tournament", ctypes.c_int), ("reps", ctypes.c_int), ("tins_init_max", ctypes.c_int),
                ("allow_merge", ctypes.c_int), ("seed", ctypes.c_uint64), ("mode", ctypes.c_int),
                ("sample_keys", ctypes.c_uint64)]


class GALog(ctypes.Structure):
    """Mirror of ``evosort_ga_log``."""
    _fields_ = [("generation", ctypes.c_int), ("best_ms", ctypes.c_float), ("mean_ms", ctypes.c_float),
                ("worst_ms", ctypes.c_float), ("evaluations", ctypes.c_int), ("best", Params)]


FitnessFn = ctypes.CFUNCTYPE(ctypes.c_float, ctypes.POINTER(Params), ctypes.c_float, ctypes.c_void_p)

CLASSES = {0: "random", 1: "skewed", 2: "narrow", 3: "few", 4: "sorted", 5: "reverse", 6: "constant",
           7: "narrow16", 8: "segmented"}
CLASS_CODE = {v: k for k, v in CLASSES.items()}
PARAM_FIELDS = ("algo", "digit_bits", "keys_per_thread", "block_size", "insertion_threshold", "rank_mode",
                "seg_block_cap", "pass_kernel", "adapt_later", "adapt_first", "seg_warp_cap", "small_cap",
                "seg_giant")


class KernelRecord(ctypes.Structure):
    """Mirror of ``evosort_kernel_record``."""
    _fields_ = [("kind", ctypes.c_int), ("pass_", ctypes.c_int), ("active", ctypes.c_int),
                ("ms", ctypes.c_float), ("bytes", ctypes.c_double), ("items", ctypes.c_uint64),
                ("rank", ctypes.c_int)]


KERNEL_KINDS = {0: "radix_histogram", 1: "radix_scan", 2: "radix_onesweep", 3: "radix_fixup",
                4: "merge_block", 5: "merge_partition", 6: "merge_pass", 7: "segmented", 8: "small", 9: "dict",
                10: "ordered", 11: "radix_count"}

_lock = threading.Lock()
_lib = None


def library():
    """The loaded ctypes handle of libevosort.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libevosort.so is not built; run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'` first")
            lib = ctypes.CDLL(_build.LIB)
            vp, sz, i, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int
            pp = ctypes.POINTER(Params)
            lib.evosort_default_params.argtypes = [pp]
            lib.evosort_default_params.restype = None
            lib.evosort_workspace_bytes.argtypes = [sz, i, i, pp]
            lib.evosort_workspace_bytes.restype = sz
            lib.evosort_resolve.argtypes = [sz, i, i, pp, pp]
            lib.evosort_resolve.restype = st
            lib.evosort_sort.argtypes = [vp, sz, i, pp]
            lib.evosort_sort_to.argtypes = [vp, vp, sz, i, pp]
            lib.evosort_sort_pairs.argtypes = [vp, vp, sz, i, pp]
            lib.evosort_sort_pairs_to.argtypes = [vp, vp, vp, vp, sz, i, pp]
            for f in (lib.evosort_sort, lib.evosort_sort_to, lib.evosort_sort_pairs, lib.evosort_sort_pairs_to):
                f.restype = st
            lib.evosort_sort_host_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                    ctypes.POINTER(sz), sz, i, pp]
            lib.evosort_sort_host_batch.restype = st
            lib.evosort_segmented_sort.argtypes = [vp, sz, vp, sz, i, pp]
            lib.evosort_segmented_sort.restype = st
            lib.evosort_segmented_workspace_bytes.argtypes = [sz, sz, i]
            lib.evosort_segmented_workspace_bytes.restype = sz
            lib.evosort_key_range.argtypes = [vp, sz, i, i, vp, vp]
            lib.evosort_key_range.restype = st
            lib.evosort_range_histogram.argtypes = [vp, sz, i, i, ctypes.c_ulonglong, i, i, vp, vp]
            lib.evosort_range_histogram.restype = st
            lib.evosort_classify.argtypes = [vp, sz, i, vp, ctypes.POINTER(ctypes.c_int)]
            lib.evosort_classify.restype = st
            lib.evosort_plan.argtypes = [vp, sz, i, vp, pp, ctypes.POINTER(ctypes.c_int)]
            lib.evosort_plan.restype = st
            lib.evosort_plan_host.argtypes = [vp, sz, i, i, pp, ctypes.POINTER(ctypes.c_int)]
            lib.evosort_plan_host.restype = st
            lib.evosort_table_set.argtypes = [i, i, i, pp, ctypes.c_float]
            lib.evosort_table_set.restype = st
            lib.evosort_table_clear.argtypes = []
            lib.evosort_table_clear.restype = None
            lib.evosort_table_size.argtypes = []
            lib.evosort_table_size.restype = sz
            lib.evosort_table_save.argtypes = [ctypes.c_char_p]
            lib.evosort_table_save.restype = st
            lib.evosort_table_load.argtypes = [ctypes.c_char_p]
            lib.evosort_table_load.restype = st
            lib.evosort_default_ga_config.argtypes = [ctypes.POINTER(GAConfig)]
            lib.evosort_default_ga_config.restype = None
            lib.evosort_tune.argtypes = [vp, sz, i, vp, ctypes.POINTER(GAConfig), vp, pp,
                                         ctypes.POINTER(ctypes.c_float), ctypes.POINTER(GALog), i]
            lib.evosort_tune.restype = st
            lib.evosort_ga_search.argtypes = [ctypes.POINTER(GAConfig), i, FitnessFn, vp, pp,
                                              ctypes.POINTER(ctypes.c_float), ctypes.POINTER(GALog), i]
            lib.evosort_ga_search.restype = st
            lib.evosort_sync.argtypes = [vp]
            lib.evosort_sync.restype = st
            lib.evosort_last_error.argtypes = []
            lib.evosort_last_error.restype = ctypes.c_char_p
            lib.evosort_profile.argtypes = [i]
            lib.evosort_profile.restype = st
            lib.evosort_profile_read.argtypes = [ctypes.POINTER(KernelRecord), sz]
            lib.evosort_profile_read.restype = sz
            lib.evosort_kernel_launches.argtypes = []
            lib.evosort_kernel_launches.restype = ctypes.c_uint64
            lib.evosort_release.argtypes = []
            lib.evosort_release.restype = st
            lib.evosort_set_wait_limit.argtypes = [ctypes.c_uint32]
            lib.evosort_set_wait_limit.restype = None
            _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        msg = library().evosort_last_error()
        raise EvoSortError(rc, msg.decode() if msg else "")


def _dtype_code(t: torch.Tensor) -> int:
    try:
        return DTYPES[t.dtype]
    except KeyError:
        raise TypeError("unsupported key dtype %s" % t.dtype) from None


def _need_cuda(*ts):
    """Every tensor on the current CUDA device (the library launches there, so
    another device's pointers would be read by the wrong GPU) and contiguous."""
    dev = None
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("tensors must be on a CUDA device")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if dev is None:
            dev = t.device
        elif t.device != dev:
            raise ValueError("tensors must be on one device (got %s and %s)" % (dev, t.device))
    if dev is not None and dev.index != torch.cuda.current_device():
        raise ValueError("tensors are on %s but the current device is cuda:%d (torch.cuda.set_device)"
                         % (dev, torch.cuda.current_device()))


def _stream_handle(stream) -> int:
    if stream is None:
        if not torch.cuda.is_available():
            return 0   # host-only calls (tables, argument checks): the legacy default stream
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(algo=None, digit_bits=0, keys_per_thread=0, block_size=0, insertion_threshold=0,
                rank_mode=0, seg_block_cap=0, stream=None, workspace: torch.Tensor | None = None,
                descending=False, pass_kernel=0, adapt_later=0, adapt_first=0, seg_warp_cap=0, small_cap=0,
                seg_giant=0) -> Params:
    p = Params()
    library().evosort_default_params(ctypes.byref(p))
    p.algo = ALGOS[algo]
    p.digit_bits = int(digit_bits or 0)
    p.keys_per_thread = int(keys_per_thread or 0)
    p.block_size = int(block_size or 0)
    p.insertion_threshold = int(insertion_threshold or 0)
    p.rank_mode = int(rank_mode or 0)
    p.seg_block_cap = int(seg_block_cap or 0)
    p.descending = 1 if descending else 0
    p.pass_kernel = int(pass_kernel or 0)
    p.adapt_later = int(adapt_later or 0)
    p.adapt_first = int(adapt_first or 0)
    p.seg_warp_cap = int(seg_warp_cap or 0)
    p.small_cap = int(small_cap or 0)
    p.seg_giant = int(seg_giant or 0)
    p.stream = _stream_handle(stream)
    if workspace is not None:
        p.workspace = workspace.data_ptr()
        p.workspace_bytes = workspace.numel() * workspace.element_size()
    return p


def sort(keys: torch.Tensor, out: torch.Tensor | None = None, *, params: Params | None = None,
         **kw) -> torch.Tensor:
    """Sorts ``keys`` (in place unless ``out`` is given) and returns the result.
    Keyword arguments are the fields of ``evosort_params`` (see make_params)."""
    _need_cuda(keys, out)
    p = params if params is not None else make_params(**kw)
    dt = _dtype_code(keys)
    lib = library()
    if out is None or out.data_ptr() == keys.data_ptr():
        _check(lib.evosort_sort(keys.data_ptr(), keys.numel(), dt, ctypes.byref(p)))
        return keys
    if out.dtype != keys.dtype or out.numel() != keys.numel():
        raise ValueError("out must match keys in dtype and size")
    _check(lib.evosort_sort_to(keys.data_ptr(), out.data_ptr(), keys.numel(), dt, ctypes.byref(p)))
    return out


def sort_pairs(keys: torch.Tensor, values: torch.Tensor, keys_out: torch.Tensor | None = None,
               values_out: torch.Tensor | None = None, *, params: Params | None = None, **kw):
    """Stable key/value sort; ``values`` are uint32.  In place unless both
    outputs are given.  Returns (keys, values)."""
    _need_cuda(keys, values, keys_out, values_out)
    if values.dtype != torch.uint32 or values.numel() != keys.numel():
        raise ValueError("values must be uint32 with one entry per key")
    p = params if params is not None else make_params(**kw)
    dt = _dtype_code(keys)
    lib = library()
    if keys_out is None and values_out is None:
        _check(lib.evosort_sort_pairs(keys.data_ptr(), values.data_ptr(), keys.numel(), dt, ctypes.byref(p)))
        return keys, values
    if keys_out is None or values_out is None:
        raise ValueError("give both keys_out and values_out, or neither")
    _check(lib.evosort_sort_pairs_to(keys.data_ptr(), values.data_ptr(), keys_out.data_ptr(),
                                     values_out.data_ptr(), keys.numel(), dt, ctypes.byref(p)))
    return keys_out, values_out


def sort_host_batch(keys: list, out: list | None = None, *, params: Params | None = None, **kw) -> list:
    """Sorts host (CPU) tensors of one dtype, each on its own, through the
    device: uploads, sorts and downloads overlap across the list.  In place
    unless ``out`` (a list of CPU tensors matching ``keys``) is given; the
    results are ready after ``sync(stream)``.  Page-locked tensors
    (``pin_memory()``) let the copies overlap the sorts."""
    keys = list(keys)
    out = keys if out is None else list(out)
    if len(out) != len(keys):
        raise ValueError("out must have one tensor per input")
    if not keys:
        return out
    dt = _dtype_code(keys[0])
    for a, b in zip(keys, out):
        if a.is_cuda or b.is_cuda:
            raise ValueError("sort_host_batch takes CPU tensors")
        if not (a.is_contiguous() and b.is_contiguous()):
            raise ValueError("tensors must be contiguous")
        if a.dtype != keys[0].dtype or b.dtype != a.dtype or b.numel() != a.numel():
            raise ValueError("all tensors must share the dtype; out must match keys in size")
    m = len(keys)
    ins = (ctypes.c_void_p * m)(*[a.data_ptr() for a in keys])
    outs = (ctypes.c_void_p * m)(*[b.data_ptr() for b in out])
    ns = (ctypes.c_size_t * m)(*[a.numel() for a in keys])
    p = params if params is not None else make_params(**kw)
    _check(library().evosort_sort_host_batch(ins, outs, ns, m, dt, ctypes.byref(p)))
    return out


def segmented_sort(keys: torch.Tensor, offsets: torch.Tensor, *, params: Params | None = None, **kw):
    """Sorts each ``keys[offsets[i]:offsets[i+1]]`` in place.  ``offsets`` is a
    device tensor of nseg + 1 int64/uint64 values starting at 0."""
    _need_cuda(keys, offsets)
    if offsets.dtype not in (torch.int64, torch.uint64):
        raise ValueError("offsets must be int64 or uint64")
    p = params if params is not None else make_params(**kw)
    _check(library().evosort_segmented_sort(keys.data_ptr(), keys.numel(), offsets.data_ptr(),
                                            offsets.numel() - 1, _dtype_code(keys), ctypes.byref(p)))
    return keys


def sync(stream=None) -> None:
    """Waits for the stream and raises if a device-side error was recorded."""
    _check(library().evosort_sync(_stream_handle(stream)))


def workspace_bytes(n: int, dtype: torch.dtype, with_values: bool = False, **kw) -> int:
    p = make_params(**kw)
    return int(library().evosort_workspace_bytes(n, DTYPES[dtype], int(with_values), ctypes.byref(p)))


def release() -> None:
    """Waits for the device and returns the library's pooled scratch memory
    on the current device to the CUDA driver (evosort_release)."""
    _check(library().evosort_release())


def set_wait_limit(polls: int) -> None:
    """Poll limit of the device-side look-back waits (0 = built-in default);
    for tests of the failure path."""
    library().evosort_set_wait_limit(int(polls))


def segmented_workspace_bytes(total: int, nseg: int, dtype: torch.dtype) -> int:
    """Scratch bytes of a batched segmented sort of total keys in nseg segments."""
    return int(library().evosort_segmented_workspace_bytes(total, nseg, DTYPES[dtype]))


def key_range(keys: torch.Tensor, descending: bool = False, stream=None) -> tuple:
    """(smallest, largest) key of a device array in the library's
    order-preserving key space, as Python ints (evosort_key_range)."""
    _need_cuda(keys)
    out = torch.empty(2, dtype=torch.int64, device=keys.device)
    _check(library().evosort_key_range(keys.data_ptr(), keys.numel(), _dtype_code(keys), int(descending),
                                       out.data_ptr(), _stream_handle(stream)))
    lo, hi = out.cpu().tolist()
    return lo & (2**64 - 1), hi & (2**64 - 1)


def range_histogram(keys: torch.Tensor, base: int, shift: int, nbins: int, descending: bool = False,
                    stream=None) -> torch.Tensor:
    """Counts (int64 device tensor of nbins) of keys with (mapped key - base)
    >> shift == b (evosort_range_histogram)."""
    _need_cuda(keys)
    counts = torch.zeros(nbins, dtype=torch.int64, device=keys.device)
    _check(library().evosort_range_histogram(keys.data_ptr(), keys.numel(), _dtype_code(keys), int(descending),
                                             ctypes.c_ulonglong(base & (2**64 - 1)), int(shift), int(nbins),
                                             counts.data_ptr(), _stream_handle(stream)))
    return counts


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(library().evosort_kernel_launches())


def profile(enable: bool) -> None:
    """Turn the library's per-launch CUDA-event instrumentation on or off."""
    _check(library().evosort_profile(int(bool(enable))))


def profile_read() -> list:
    """Per-launch records since the last read: dicts with kind, pass, active,
    ms (device time between the events around the launch), bytes
    (algorithmic traffic of the launch), items and rank (the ranking variant
    of a radix pass launch under adaptive ranking, else 0)."""
    lib = library()
    cap = 1 << 16
    buf = (KernelRecord * cap)()
    n = int(lib.evosort_profile_read(buf, cap))
    return [{"kind": KERNEL_KINDS.get(r.kind, r.kind), "pass": r.pass_, "active": bool(r.active),
             "ms": float(r.ms), "bytes": float(r.bytes), "items": int(r.items), "rank": int(r.rank)}
            for r in buf[:min(n, cap)]]


def params_dict(p: Params) -> dict:
    """The tunable fields of a Params struct as a dict."""
    return {f: int(getattr(p, f)) for f in PARAM_FIELDS}


def classify(keys: torch.Tensor, stream=None) -> str:
    """Distribution class of ``keys`` from a strided sample (synchronises)."""
    _need_cuda(keys)
    c = ctypes.c_int(0)
    _check(library().evosort_classify(keys.data_ptr(), keys.numel(), _dtype_code(keys), _stream_handle(stream),
                                      ctypes.byref(c)))
    return CLASSES[c.value]


def plan(keys: torch.Tensor, stream=None):
    """(params dict, class) the dispatcher would use for ``keys``."""
    _need_cuda(keys)
    p = Params()
    c = ctypes.c_int(0)
    _check(library().evosort_plan(keys.data_ptr(), keys.numel(), _dtype_code(keys), _stream_handle(stream),
                                  ctypes.byref(p), ctypes.byref(c)))
    return params_dict(p), CLASSES[c.value]


def resolve(n: int, dtype: torch.dtype, with_values: bool = False, **kw) -> dict:
    """Every parameter a sort of n keys would run with (defaults resolved;
    no table lookup); keyword arguments as for make_params."""
    out = Params()
    p = make_params(**kw)
    _check(library().evosort_resolve(n, DTYPES[dtype], int(with_values), ctypes.byref(p), ctypes.byref(out)))
    return params_dict(out)


def plan_host(keys: torch.Tensor, descending: bool = False):
    """(params dict, class) for keys in host memory, classified from a
    strided sample read on the host (no device access)."""
    if keys.is_cuda:
        raise ValueError("plan_host takes a CPU tensor")
    if not keys.is_contiguous():
        raise ValueError("tensors must be contiguous")
    p = Params()
    c = ctypes.c_int(0)
    _check(library().evosort_plan_host(keys.data_ptr(), keys.numel(), _dtype_code(keys), int(descending),
                                       ctypes.byref(p), ctypes.byref(c)))
    return params_dict(p), CLASSES[c.value]


def table_set(dtype: torch.dtype, size_bucket: int, cls: str, params: dict, ms: float = 0.0) -> None:
    p = make_params(**{k: v for k, v in params.items() if k != "algo"}, algo=params.get("algo", 0))
    _check(library().evosort_table_set(DTYPES[dtype], int(size_bucket), CLASS_CODE[cls], ctypes.byref(p),
                                       float(ms)))


def table_clear() -> None:
    library().evosort_table_clear()


def table_size() -> int:
    return int(library().evosort_table_size())


def table_save(path: str) -> None:
    _check(library().evosort_table_save(path.encode()))


def table_load(path: str) -> None:
    _check(library().evosort_table_load(path.encode()))


def tune(sample: torch.Tensor, expected: torch.Tensor | None = None, stream=None, **ga):
    """Runs the genetic algorithm on one device sample.  Returns
    (best params dict, best ms, per-generation log as a list of dicts).
    ``ga`` overrides fields of the default GA configuration."""
    _need_cuda(sample, expected)
    lib = library()
    cfg = GAConfig()
    lib.evosort_default_ga_config(ctypes.byref(cfg))
    for k, v in ga.items():
        setattr(cfg, k, v)
    best = Params()
    best_ms = ctypes.c_float(0)
    logs = (GALog * max(cfg.generations, 1))()
    _check(lib.evosort_tune(sample.data_ptr(), sample.numel(), _dtype_code(sample),
                            expected.data_ptr() if expected is not None else None, ctypes.byref(cfg),
                            _stream_handle(stream), ctypes.byref(best), ctypes.byref(best_ms), logs,
                            cfg.generations))
    log = [{"generation": g.generation, "best_ms": g.best_ms, "mean_ms": g.mean_ms, "worst_ms": g.worst_ms,
            "evaluations": g.evaluations, "best": params_dict(g.best)} for g in logs[:cfg.generations]]
    return params_dict(best), float(best_ms.value), log


def ga_search(fitness, key_bytes: int = 8, **ga):
    """The GA loop with a Python fitness function ``fitness(params_dict,
    best_so_far_ms) -> ms`` (negative = failed genome).  Returns (best params
    dict, best ms, log)."""
    lib = library()
    cfg = GAConfig()
    lib.evosort_default_ga_config(ctypes.byref(cfg))
    for k, v in ga.items():
        setattr(cfg, k, v)

    def cb(pp, best_so_far, _ctx):
        return float(fitness(params_dict(pp.contents), float(best_so_far)))

    fn = FitnessFn(cb)
    best = Params()
    best_ms = ctypes.c_float(0)
    logs = (GALog * max(cfg.generations, 1))()
    _check(lib.evosort_ga_search(ctypes.byref(cfg), int(key_bytes), fn, None, ctypes.byref(best),
                                 ctypes.byref(best_ms), logs, cfg.generations))
    log = [{"generation": g.generation, "best_ms": g.best_ms, "mean_ms": g.mean_ms, "worst_ms": g.worst_ms,
            "evaluations": g.evaluations, "best": params_dict(g.best)} for g in logs[:cfg.generations]]
    return params_dict(best), float(best_ms.value), log
