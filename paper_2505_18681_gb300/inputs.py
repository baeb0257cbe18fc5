"""Seeded synthetic inputs for the sort workloads.

This module only draws numbers; it holds none of the sort's arithmetic, and
both the CUDA path's tests and the CPU oracle's tests take their inputs from
it.  Every draw is counter based: element ``i`` of stream ``s`` under seed
``seed`` is the ``i``-th output of SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) started from a state
derived from ``(seed, s)``.  The same code runs on any torch device, so CPU and
GPU draws of the integer distributions are identical; float distributions may
differ in the last bit between devices, which does not matter because the
oracle always sorts a host copy of the exact device input.

Distributions (names used by the tests, the benchmark and the tuner):

* ``uniform``        full range of the dtype (random bit patterns for ints)
* ``uniform_paper``  integers uniform in [-1e9, 1e9] (the paper's workload)
* ``gaussian``       N(0, 1e6) rounded half-to-even
* ``sorted`` / ``reverse``   x[i] = MIN + i * floor(2^w / n), or its reverse
* ``nearly_sorted``  ``sorted`` with n // 100 swaps of disjoint random pairs
* ``distinct16``     each element one of 16 seeded full-range values
* ``zipf``           rank in [1, 1e6] with P(k) proportional to k^-1.2
* ``equal``          one seeded value everywhere
* ``uniform1000``    integers uniform in [0, 1000)
* ``float_mix``      float64 uniform in [-1e6, 1e6], 1% of positions copied
  from other positions, then 0.1% each of -0.0, +0.0, +qNaN, -qNaN

The paper's own nine integer distributions (its Section 5 data-distribution
tests), mapped to [-1e9, 1e9] as the paper describes and truncated toward
zero to integers; counter-based draws stand in for NumPy's generator, so the
shapes match and the exact values do not:

* ``paper_uniform``        integers uniform in [-1e9, 1e9)
* ``paper_normal``         N(0, 1e8) clipped to [-1e9, 1e9]
* ``paper_exponential``    Exp(scale 1e9) clipped to [0, 2e9], minus 1e9
* ``paper_power``          power law with a = 0.5 (u^(1/a)) scaled to [-1e9, 1e9]
* ``paper_beta``           Beta(2, 5) scaled to [-1e9, 1e9]
* ``paper_sparse``         zero, except each position with probability 0.1 is
  a uniform integer in [-1e9, 1e9)
* ``paper_clustered``      one of 10 evenly spaced centres in [-1e9, 1e9] plus
  N(0, 1e8), clipped
* ``paper_nearly_sorted``  the evenly spaced ramp from -1e9 to 1e9, each
  position replaced with probability 0.1 by a uniform integer
* ``paper_duplicates``     each element one of n // 10 seeded uniform integers

A stand-in for the paper's real-data test (the Friendster edge list's
endpoint column, which is not available here):

* ``friendster_like``  node ids in [101, 124,836,179] with a heavy-tailed
  frequency: node rank k = floor(M u^3) over M = 65,608,366 nodes (density
  proportional to k^(-2/3)), mapped to an id by a fixed bijection
  k -> 101 + (k * 2654435761 mod 124,836,078), so frequent ids spread over
  the range

Distributions drawn through log / cos (``gaussian``, ``paper_normal``,
``paper_exponential``, ``paper_beta``, ``paper_clustered``) may differ in a
rare last integer step between devices; every test sorts the exact device
input, so this never matters.
"""
from __future__ import annotations

import math

import torch

_MASK64 = (1 << 64) - 1


def _s64(v: int) -> int:
    v &= _MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)

_CHUNK = 1 << 26

DISTRIBUTIONS = ("uniform", "gaussian", "sorted", "reverse", "nearly_sorted",
                 "distinct16", "zipf", "equal", "uniform1000")

PAPER_DISTRIBUTIONS = ("paper_uniform", "paper_normal", "paper_exponential", "paper_power", "paper_beta",
                       "paper_sparse", "paper_clustered", "paper_nearly_sorted", "paper_duplicates")

FRIENDSTER_N = 3_612_134_270        # endpoints in the paper's real-data test
_FRIENDSTER_NODES = 65_608_366
_FRIENDSTER_LO, _FRIENDSTER_HI = 101, 124_836_179

_STREAM_ID = {name: i + 1 for i, name in enumerate(
    DISTRIBUTIONS + ("uniform_paper", "float_mix", "seglen", "segkeys", "aux") + PAPER_DISTRIBUTIONS +
    ("friendster_like",))}


def _lsr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _lsr(z, 30)) * _C1
    z = (z ^ _lsr(z, 27)) * _C2
    return z ^ _lsr(z, 31)


def _mix_int(x: int) -> int:
    z = x & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_state(seed: int, stream: int) -> int:
    """Start state of stream ``stream`` under ``seed`` (a SplitMix64 output)."""
    return _s64(_mix_int(_mix_int(seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) ^ (stream + 1)))


def raw64(state: int, start: int, count: int, device) -> torch.Tensor:
    """SplitMix64 outputs ``start .. start+count-1`` of a stream, as int64."""
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return _mix(i * _GOLDEN + state)


def unit_double(r: torch.Tensor) -> torch.Tensor:
    """53-bit uniform double in [0, 1) from int64 random bits."""
    return _lsr(r, 11).to(torch.float64) * (2.0 ** -53)


def _bounded(r: torch.Tensor, m: int) -> torch.Tensor:
    """Integer in [0, m) from random bits (63-bit remainder; bias < m / 2^63)."""
    return _lsr(r, 1) % m


_INT_DTYPES = {torch.int32: 32, torch.int64: 64, torch.uint32: 32, torch.uint64: 64}


def _as_dtype(x64: torch.Tensor, dtype: torch.dtype) -> torch.Tensor:
    """Reinterpret the low bits of int64 values as ``dtype`` (two's complement)."""
    if dtype == torch.int64:
        return x64
    if dtype == torch.uint64:
        return x64.view(torch.uint64) if hasattr(torch, "uint64") else x64
    lo = x64 & 0xFFFFFFFF
    lo = torch.where(lo >= (1 << 31), lo - (1 << 32), lo).to(torch.int32)
    if dtype == torch.int32:
        return lo
    return lo.view(torch.uint32)


def _fill(n: int, dtype: torch.dtype, device, fn) -> torch.Tensor:
    """Allocate the output and fill it chunk by chunk with ``fn(start, count)``
    (which returns int64 bit patterns or float64 values)."""
    out = torch.empty(n, dtype=dtype, device=device)
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        v = fn(s, c)
        if dtype.is_floating_point:
            out[s:s + c] = v.to(dtype)
        else:
            out[s:s + c] = _as_dtype(v, dtype)
    return out


def _signed_min(bits: int, dtype) -> int:
    return 0 if dtype in (torch.uint32, torch.uint64) else -(1 << (bits - 1))


def generate(dist: str, n: int, dtype=torch.int64, seed: int = 42, device="cpu") -> torch.Tensor:
    """Seeded synthetic keys of distribution ``dist``; see the module docstring."""
    st = stream_state(seed, _STREAM_ID[dist])
    if dist == "float_mix":
        return _float_mix(n, dtype, seed, device)
    if dtype.is_floating_point:
        return _float_dist(dist, n, dtype, st, device)
    bits = _INT_DTYPES[dtype]
    lo = _signed_min(bits, dtype)
    if dist == "uniform":
        return _fill(n, dtype, device, lambda s, c: raw64(st, s, c, device))
    if dist == "uniform_paper":
        return _fill(n, dtype, device,
                     lambda s, c: _bounded(raw64(st, s, c, device), 2_000_000_001) - 1_000_000_000)
    if dist == "uniform1000":
        return _fill(n, dtype, device, lambda s, c: _bounded(raw64(st, s, c, device), 1000))
    if dist == "gaussian":
        def g(s, c):
            u1 = unit_double(raw64(st, s, c, device))
            u2 = unit_double(raw64(stream_state(seed, 99), s, c, device))
            z = torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)
            return torch.round(z * 1e6).to(torch.int64)
        return _fill(n, dtype, device, g)
    if dist in ("sorted", "reverse", "nearly_sorted"):
        step = _s64((1 << bits) // max(n, 2))
        def ramp(s, c):
            i = torch.arange(s, s + c, dtype=torch.int64, device=device)
            if dist == "reverse":
                i = (n - 1) - i
            return i * step + lo
        x = _fill(n, dtype, device, ramp)
        if dist == "nearly_sorted":
            _disjoint_swaps(x, n // 100, seed, device)
        return x
    if dist == "distinct16":
        vals = raw64(st, 0, 16, device)
        st2 = stream_state(seed, _STREAM_ID["aux"])
        return _fill(n, dtype, device, lambda s, c: vals[_bounded(raw64(st2, s, c, device), 16)])
    if dist == "zipf":
        k = torch.arange(1, 1_000_001, dtype=torch.float64, device=device)
        cdf = torch.cumsum(k ** -1.2, 0)
        cdf = cdf / cdf[-1]
        return _fill(n, dtype, device,
                     lambda s, c: torch.clamp(torch.searchsorted(cdf, unit_double(raw64(st, s, c, device)),
                                                                 right=True), max=999_999) + 1)
    if dist == "equal":
        v = raw64(st, 0, 1, "cpu").item()
        return _fill(n, dtype, device,
                     lambda s, c: torch.full((c,), v, dtype=torch.int64, device=device))
    if dist in PAPER_DISTRIBUTIONS:
        return _fill(n, dtype, device, _paper_fn(dist, n, seed, st, device))
    if dist == "friendster_like":
        span = _FRIENDSTER_HI - _FRIENDSTER_LO   # 124,836,078; the multiplier is odd and coprime to it
        def fr(s, c):
            k = torch.floor(_FRIENDSTER_NODES * unit_double(raw64(st, s, c, device)) ** 3).to(torch.int64)
            return _FRIENDSTER_LO + (k * 2654435761) % span
        return _fill(n, dtype, device, fr)
    raise ValueError("unknown distribution %r" % dist)


def raw64_at(state: int, idx: torch.Tensor) -> torch.Tensor:
    """SplitMix64 outputs at arbitrary positions ``idx`` (int64) of a stream."""
    return _mix((idx + 1) * _GOLDEN + state)


def _paper_fn(dist, n, seed, st, device):
    """Chunk filler for the paper's nine distributions (values as int64)."""
    def sub(j):   # independent sub-streams of this distribution
        return stream_state(seed, 1000 * _STREAM_ID[dist] + j)

    def u(j, s, c):
        return unit_double(raw64(sub(j), s, c, device))

    def randint(j, s, c):   # uniform in [-1e9, 1e9)
        return _bounded(raw64(sub(j), s, c, device), 2_000_000_000) - 1_000_000_000

    def normal(j, s, c):
        return torch.sqrt(-2.0 * torch.log1p(-u(j, s, c))) * torch.cos(2.0 * math.pi * u(j + 1, s, c))

    def to_int(x):
        return torch.trunc(x).to(torch.int64)

    if dist == "paper_uniform":
        return lambda s, c: randint(0, s, c)
    if dist == "paper_normal":
        return lambda s, c: to_int(torch.clamp(normal(0, s, c) * 1e8, -1e9, 1e9))
    if dist == "paper_exponential":
        return lambda s, c: to_int(torch.clamp(-torch.log1p(-u(0, s, c)) * 1e9, 0.0, 2e9) - 1e9)
    if dist == "paper_power":
        return lambda s, c: to_int(u(0, s, c) ** 2 * 2e9 - 1e9)
    if dist == "paper_beta":
        def beta(s, c):
            # Beta(2, 5) = G2 / (G2 + G5), Gamma(k) a sum of k unit exponentials
            e = [-torch.log1p(-u(j, s, c)) for j in range(7)]
            g2 = e[0] + e[1]
            g5 = e[2] + e[3] + e[4] + e[5] + e[6]
            return to_int(g2 / (g2 + g5) * 2e9 - 1e9)
        return beta
    if dist == "paper_sparse":
        return lambda s, c: torch.where(u(0, s, c) < 0.1, randint(1, s, c), torch.zeros_like(randint(1, s, c)))
    if dist == "paper_clustered":
        def clustered(s, c):
            k = _bounded(raw64(sub(0), s, c, device), 10).to(torch.float64)
            centre = -1e9 + k * (2e9 / 9.0)
            return to_int(torch.clamp(centre + normal(1, s, c) * 1e8, -1e9, 1e9))
        return clustered
    if dist == "paper_nearly_sorted":
        def nearly(s, c):
            i = torch.arange(s, s + c, dtype=torch.float64, device=device)
            ramp = to_int(-1e9 + i * (2e9 / max(n - 1, 1)))
            return torch.where(u(0, s, c) < 0.1, randint(1, s, c), ramp)
        return nearly
    if dist == "paper_duplicates":
        m = max(n // 10, 1)
        def dup(s, c):
            k = _bounded(raw64(sub(0), s, c, device), m)
            return _bounded(raw64_at(sub(1), k), 2_000_000_000) - 1_000_000_000
        return dup
    raise ValueError(dist)


def _disjoint_swaps(x: torch.Tensor, m: int, seed: int, device) -> None:
    """Apply ``m`` swaps of disjoint random position pairs to ``x`` in place.
    Positions: one per stripe of width n // (2m); stripes paired by a seeded
    random permutation, so no position is touched twice."""
    n = x.numel()
    if m <= 0 or n < 2 * m:
        return
    if x.dtype in (torch.uint32, torch.uint64):
        x = x.view(torch.int32 if x.dtype == torch.uint32 else torch.int64)
    width = n // (2 * m)
    st = stream_state(seed, _STREAM_ID["aux"])
    off = _bounded(raw64(st, 0, 2 * m, device), width)
    pos = torch.arange(2 * m, dtype=torch.int64, device=device) * width + off
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    perm = torch.randperm(2 * m, generator=g).to(device)
    a = pos[perm[0::2]]
    b = pos[perm[1::2]]
    xa = x[a].clone()
    x[a] = x[b]
    x[b] = xa


def _float_dist(dist, n, dtype, st, device):
    if dist in ("uniform", "uniform_paper"):
        return _fill(n, dtype, device,
                     lambda s, c: unit_double(raw64(st, s, c, device)) * 2e6 - 1e6)
    raise ValueError("distribution %r is integer-only" % dist)


def _float_mix(n, dtype, seed, device):
    """Float workload: uniform [-1e6, 1e6], 1% duplicates, signed zeros and
    NaNs of both signs (bit patterns 0x7FF8.. and 0xFFF8..)."""
    st = stream_state(seed, _STREAM_ID["float_mix"])
    x = _fill(n, torch.float64, device, lambda s, c: unit_double(raw64(st, s, c, device)) * 2e6 - 1e6)
    aux = stream_state(seed, _STREAM_ID["aux"])
    m = n // 100
    if m:
        p = torch.arange(m, dtype=torch.int64, device=device) * 100 + _bounded(raw64(aux, 0, m, device), 100)
        q = _bounded(raw64(aux, m, m, device), n)
        x[p] = x[q].clone()
    k = n // 250
    if k:
        p = torch.arange(k, dtype=torch.int64, device=device) * 250 + _bounded(raw64(aux, 2 * m, k, device), 250)
        xb = x.view(torch.int64)
        specials = torch.tensor([_s64(0x8000000000000000), 0, 0x7FF8000000000000,
                                 _s64(0xFFF8000000000000)], dtype=torch.int64, device=device)
        xb[p] = specials[torch.arange(k, device=device) % 4]
    if dtype == torch.float32:
        return x.to(torch.float32)
    return x


def segment_lengths(nseg: int, lo: int = 16, hi: int = 1_000_000, seed: int = 42) -> torch.Tensor:
    """Log-uniform segment lengths floor(exp(U(ln lo, ln hi))) on the CPU."""
    st = stream_state(seed, _STREAM_ID["seglen"])
    u = unit_double(raw64(st, 0, nseg, "cpu"))
    ln = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return torch.clamp(torch.floor(ln).to(torch.int64), lo, hi)


def _segmented_fn(lengths: torch.Tensor, dtype, seed: int, device):
    """Chunk filler of the segmented batch: the key at global position i
    depends only on i, its segment and its place in the segment."""
    lengths = lengths.to(torch.int64).cpu()
    offsets = torch.zeros(lengths.numel() + 1, dtype=torch.int64)
    offsets[1:] = torch.cumsum(lengths, 0)
    bits = _INT_DTYPES[dtype]
    lo = _signed_min(bits, dtype)
    st = stream_state(seed, _STREAM_ID["segkeys"])
    aux = stream_state(seed, _STREAM_ID["aux"])
    offs_dev = offsets.to(device)
    lens_dev = lengths.to(device)

    def fn(s, c):
        i = torch.arange(s, s + c, dtype=torch.int64, device=device)
        seg = torch.searchsorted(offs_dev, i, right=True) - 1
        local = i - offs_dev[seg]
        r = raw64(st, s, c, device)
        step = ((1 << (bits - 2)) // torch.clamp(lens_dev[seg], min=1)) * 4   # ~2^bits / len, in int64
        ramp = local * step + lo
        replace = _bounded(raw64(aux, s, c, device), 100) == 0
        odd = (seg & 1) == 1
        return torch.where(odd & ~replace, ramp, r)

    return fn, offsets


def segmented_keys(lengths: torch.Tensor, dtype=torch.int32, seed: int = 42, device="cpu"):
    """Keys for a batched segmented sort: even segments uniform full range, odd
    segments an ascending ramp with 1% of positions replaced by uniform random
    values.  Returns (keys, offsets) with offsets as int64 of length nseg+1."""
    fn, offsets = _segmented_fn(lengths, dtype, seed, device)
    return _fill(int(offsets[-1]), dtype, device, fn), offsets


def segmented_keys_range(lengths: torch.Tensor, start: int, stop: int, dtype=torch.int32, seed: int = 42,
                         device="cpu") -> torch.Tensor:
    """The keys at global positions [start, stop) of segmented_keys(lengths,
    dtype, seed), generated without the rest of the batch."""
    fn, _ = _segmented_fn(lengths, dtype, seed, device)
    return _fill(stop - start, dtype, device, lambda s, c: fn(start + s, c))
