"""EvoSort CPU oracle — test infrastructure only.

Python loader for ``oracle/oracle.c`` (plain single-threaded C, built with gcc
into ``oracle/_build/``).  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the GPU library never
does, and the two share no code.

Functions take and return numpy arrays:

* ``radix_sort(keys, values=None)``  — O1, LSD radix with 8-bit digits
  (Algorithms 4a/4b of the paper);
* ``merge_sort(keys, values=None, chunk_size=32)`` — O2, bottom-up mergesort
  with insertion-sorted base chunks (Algorithm 3);
* ``segmented_sort(keys, offsets)`` — O1 per segment;
* ``ordered_bits(raw_bits, dtype)`` — the total-order map on key bits;
* ``parallel_radix_sort(keys, threads=0)`` — the CPU baseline, not an oracle:
  the paper's multithreaded radix sort shape (per-thread histograms and
  thread-wise offsets, Algorithms 4a/4b) on the host cores
  (``oracle/cpu_parallel.c``, checked against O1 in the tests).

Parity status: pinned (see ``tests/test_oracle.py``): brute force over all
permutations of tiny inputs, a selection sort written from the definition of
the total order, numpy's stable sort for integer keys, the float order spelled
out by category, and invariants (sortedness, permutation, stability).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

_DT_CODE = {
    np.dtype(np.int32): 0,
    np.dtype(np.int64): 1,
    np.dtype(np.uint32): 2,
    np.dtype(np.uint64): 3,
    np.dtype(np.float32): 4,
    np.dtype(np.float64): 5,
}

_PAR_SRC = os.path.join(_HERE, "cpu_parallel.c")
_PAR_LIB_PATH = os.path.join(_BUILD, "libcpu_parallel.so")

_lock = threading.Lock()
_lib = None
_par_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    par_stale = force or not os.path.exists(_PAR_LIB_PATH) or (
        os.path.getmtime(_PAR_LIB_PATH) < os.path.getmtime(_PAR_SRC))
    if par_stale:
        tmp = _PAR_LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _PAR_SRC])
        os.replace(tmp, _PAR_LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
            lib.oracle_radix_sort.argtypes = [vp, vp, sz, i, vp, vp]
            lib.oracle_radix_sort.restype = i
            lib.oracle_merge_sort.argtypes = [vp, vp, sz, i, sz, vp, vp]
            lib.oracle_merge_sort.restype = i
            lib.oracle_segmented_sort.argtypes = [vp, vp, sz, i, vp]
            lib.oracle_segmented_sort.restype = i
            lib.oracle_ordered_bits.argtypes = [ctypes.c_uint64, i]
            lib.oracle_ordered_bits.restype = ctypes.c_uint64
            lib.oracle_set_fault.argtypes = [i]
            lib.oracle_set_fault.restype = None
            _lib = lib
    return _lib


def _code(keys: np.ndarray) -> int:
    try:
        return _DT_CODE[keys.dtype]
    except KeyError:
        raise TypeError("unsupported key dtype %s" % keys.dtype) from None


def _ptr(a):
    return None if a is None else a.ctypes.data


def radix_sort(keys: np.ndarray, values: np.ndarray | None = None):
    """O1: returns sorted keys (and the values moved with them, if given)."""
    lib = _load()
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    vin = vout = None
    if values is not None:
        vin = np.ascontiguousarray(values, dtype=np.uint32)
        if vin.shape != keys.shape:
            raise ValueError("values must match keys")
        vout = np.empty_like(vin)
    rc = lib.oracle_radix_sort(_ptr(keys), _ptr(vin), keys.size, _code(keys), _ptr(out), _ptr(vout))
    if rc:
        raise MemoryError("oracle_radix_sort failed (%d)" % rc)
    return out if values is None else (out, vout)


def merge_sort(keys: np.ndarray, values: np.ndarray | None = None, chunk_size: int = 32):
    """O2: bottom-up mergesort with insertion-sorted chunks of ``chunk_size``."""
    lib = _load()
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    vin = vout = None
    if values is not None:
        vin = np.ascontiguousarray(values, dtype=np.uint32)
        vout = np.empty_like(vin)
    rc = lib.oracle_merge_sort(_ptr(keys), _ptr(vin), keys.size, _code(keys), int(chunk_size),
                               _ptr(out), _ptr(vout))
    if rc:
        raise MemoryError("oracle_merge_sort failed (%d)" % rc)
    return out if values is None else (out, vout)


def segmented_sort(keys: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    """O1 applied to each segment ``[offsets[i], offsets[i+1])``."""
    lib = _load()
    keys = np.ascontiguousarray(keys)
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    out = keys.copy()
    rc = lib.oracle_segmented_sort(_ptr(keys), _ptr(offs), offs.size - 1, _code(keys), _ptr(out))
    if rc:
        raise ValueError("oracle_segmented_sort failed (%d)" % rc)
    return out


def ordered_bits(raw: int, dtype) -> int:
    """The total-order map applied to one key's raw bit pattern."""
    return int(_load().oracle_ordered_bits(int(raw), _DT_CODE[np.dtype(dtype)]))


def set_fault(code: int) -> None:
    """Plant a known mistake in the oracle (self-tests of the pins only)."""
    _load().oracle_set_fault(int(code))


def parallel_radix_sort(keys: np.ndarray, threads: int = 0):
    """CPU baseline: returns (sorted keys, threads used).  threads <= 0 uses
    every online CPU."""
    global _par_lib
    with _lock:
        if _par_lib is None:
            build()
            lib = ctypes.CDLL(_PAR_LIB_PATH)
            lib.cpu_parallel_radix_sort.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                                    ctypes.c_int, ctypes.c_int]
            lib.cpu_parallel_radix_sort.restype = ctypes.c_int
            _par_lib = lib
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    used = _par_lib.cpu_parallel_radix_sort(_ptr(keys), _ptr(out), keys.size, _code(keys), int(threads))
    if used < 0:
        raise MemoryError("cpu_parallel_radix_sort failed")
    return out, used
