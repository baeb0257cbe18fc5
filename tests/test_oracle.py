"""Pins for the CPU oracle (no GPU).

The oracle's result has a plain definition (a stable sort under a stated total
order), so it is pinned by things that do not use its own code:

* a selection sort written in Python from the definition, with the float
  order spelled out by category rather than through the bit map;
* brute force: every permutation of tiny inputs must give the same output;
* numpy's stable sort for integer keys (the paper's own check is equality with
  np.sort, Section 5, validation methodology);
* hand-written golden orders (tests/golden/);
* invariants: sorted, a permutation of the input (counts of bit patterns),
  stable for equal keys; all-equal, sorted and reversed special cases.

The last test plants each of several plausible mistakes in the oracle and
checks that some pin fails for each.
"""
import collections
import itertools
import math
import os
import struct

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INT_DTYPES = [np.int32, np.int64, np.uint32, np.uint64]
ALL_DTYPES = INT_DTYPES + [np.float32, np.float64]


# --------------------------------------------------------------------------
# Definition of the order, written independently of the oracle's bit map.
# --------------------------------------------------------------------------
def _float_fields(bits, dtype):
    if np.dtype(dtype) == np.float64:
        sign, exp, man = bits >> 63, (bits >> 52) & 0x7FF, bits & ((1 << 52) - 1)
        emax = 0x7FF
        val = struct.unpack("<d", struct.pack("<Q", bits))[0]
    else:
        sign, exp, man = bits >> 31, (bits >> 23) & 0xFF, bits & ((1 << 23) - 1)
        emax = 0xFF
        val = struct.unpack("<f", struct.pack("<I", bits))[0]
    return sign, exp, man, emax, val


def definition_key(bits, dtype):
    """Rank tuple of one key under the library's total order."""
    dtype = np.dtype(dtype)
    if dtype.kind in "iu":
        w = dtype.itemsize * 8
        if dtype.kind == "i" and bits >= (1 << (w - 1)):
            return (bits - (1 << w),)
        return (bits,)
    sign, exp, man, emax, val = _float_fields(bits, dtype)
    if exp == emax and man != 0:                      # NaN
        return (7, -man) if sign else (6, man)
    if math.isinf(val):
        return (5,) if val > 0 else (0,)
    if val == 0.0:
        return (2,) if sign else (3,)
    return (1, val) if val < 0 else (4, val)


def as_bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def definition_sort(keys, values=None):
    """Stable selection sort from the definition (tiny inputs only)."""
    bits = [int(b) for b in as_bits(keys)]
    idx = list(range(len(bits)))
    out = []
    while idx:
        best = idx[0]
        for j in idx[1:]:
            if definition_key(bits[j], keys.dtype) < definition_key(bits[best], keys.dtype):
                best = j
        out.append(best)
        idx.remove(best)
    order = np.array(out, dtype=np.int64)
    k = keys[order] if len(order) else keys[:0]
    if values is None:
        return k
    return k, values[order]


def check_invariants(inp, out, vin=None, vout=None):
    """Sorted under the definition, a permutation of the input, stable."""
    bi, bo = as_bits(inp), as_bits(out)
    assert collections.Counter(bi.tolist()) == collections.Counter(bo.tolist())
    ranks = [definition_key(int(b), inp.dtype) for b in bo]
    for a, b in zip(ranks, ranks[1:]):
        assert a <= b
    if vin is not None:
        assert sorted(vout.tolist()) == sorted(vin.tolist())
        for i in range(1, len(out)):
            if bo[i] == bo[i - 1]:
                assert vout[i] > vout[i - 1]
        # each (key, value) pair of the output exists in the input
        pairs_in = collections.Counter(zip(bi.tolist(), vin.tolist()))
        assert pairs_in == collections.Counter(zip(bo.tolist(), vout.tolist()))


def alphabet(dtype):
    dtype = np.dtype(dtype)
    if dtype == np.int32:
        return np.array([-1, 0, 1, -2**31, 2**31 - 1], dtype=dtype)
    if dtype == np.int64:
        return np.array([-1, 0, 1, -2**63, 2**63 - 1], dtype=dtype)
    if dtype.kind == "u":
        return np.array([0, 1, 255, 256, np.iinfo(dtype).max], dtype=dtype)
    f = np.array([-np.inf, -0.0, 0.0, 1.5, np.inf, np.nan, -np.nan], dtype=dtype)
    # make the second NaN a negative quiet NaN explicitly
    b = as_bits(f).copy()
    b[6] = b[5] | (1 << (8 * dtype.itemsize - 1))
    return b.view(dtype)


# --------------------------------------------------------------------------
# Brute force over permutations of tiny inputs.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ALL_DTYPES, ids=lambda d: np.dtype(d).name)
def test_brute_force_permutations(dtype):
    al = alphabet(dtype)
    rng = np.random.default_rng(7)
    cases = []
    for n in range(0, 5):
        for combo in itertools.combinations_with_replacement(range(len(al)), n):
            cases.append(list(combo))
    for n in (5, 6):
        for _ in range(6):
            cases.append(rng.integers(0, len(al), n).tolist())
    for combo in cases:
        base = al[np.array(combo, dtype=np.int64)] if combo else al[:0]
        expect_bits = as_bits(definition_sort(base))
        seen = set()
        for perm in itertools.permutations(range(len(combo))):
            p = np.array(perm, dtype=np.int64)
            x = base[p] if len(p) else base
            key = as_bits(x).tobytes()
            if key in seen:
                continue
            seen.add(key)
            o1 = oracle.radix_sort(x)
            o2 = oracle.merge_sort(x, chunk_size=2)
            assert np.array_equal(as_bits(o1), expect_bits), (combo, perm)
            assert np.array_equal(as_bits(o2), expect_bits), (combo, perm)


@pytest.mark.parametrize("dtype", ALL_DTYPES, ids=lambda d: np.dtype(d).name)
def test_brute_force_pairs_stability(dtype):
    """Every permutation of tiny inputs, values = input index: the pairs output
    equals the stable selection sort from the definition."""
    al = alphabet(dtype)
    rng = np.random.default_rng(11)
    for n in range(1, 7):
        for _ in range(5):
            base = al[rng.integers(0, 3, n)]          # few symbols -> many ties
            for perm in itertools.islice(itertools.permutations(range(n)), 60):
                x = base[np.array(perm)]
                v = np.arange(n, dtype=np.uint32)
                ek, ev = definition_sort(x, v)
                for k, vv in (oracle.radix_sort(x, v), oracle.merge_sort(x, v, chunk_size=3)):
                    assert np.array_equal(as_bits(k), as_bits(ek))
                    assert np.array_equal(vv, ev)


# --------------------------------------------------------------------------
# Library special case: numpy's stable sort on integers.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", INT_DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 255, 256, 257, 1000, 4099, 65537])
def test_matches_numpy_stable(dtype, n):
    rng = np.random.default_rng(n)
    info = np.iinfo(dtype)
    for spread in (None, 7, 1000):
        if spread is None:
            x = rng.integers(info.min, info.max, n, dtype=dtype, endpoint=True)
        else:
            x = rng.integers(0, spread, n).astype(dtype)
        v = np.arange(n, dtype=np.uint32)
        ek = np.sort(x, kind="stable")
        ev = np.argsort(x, kind="stable").astype(np.uint32)
        k1, v1 = oracle.radix_sort(x, v)
        k2, v2 = oracle.merge_sort(x, v, chunk_size=32)
        assert np.array_equal(k1, ek) and np.array_equal(v1, ev)
        assert np.array_equal(k2, ek) and np.array_equal(v2, ev)
        assert np.array_equal(oracle.radix_sort(x), ek)


def test_paper_workload_shape_matches_numpy():
    """int32 uniform in [-1e9, 1e9] (the paper's workload), checked the way the
    paper checks it: equal to np.sort of a copy."""
    rng = np.random.default_rng(42)
    x = rng.integers(-10**9, 10**9, 200_003, dtype=np.int32, endpoint=True)
    assert np.array_equal(oracle.radix_sort(x), np.sort(x.copy()))
    assert np.array_equal(oracle.merge_sort(x, chunk_size=64), np.sort(x.copy()))


# --------------------------------------------------------------------------
# Golden orders.
# --------------------------------------------------------------------------
def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("name,dtype,udt", [("float_order_f64.txt", np.float64, np.uint64),
                                            ("float_order_f32.txt", np.float32, np.uint32)])
def test_golden_float_order(name, dtype, udt):
    rows = _read_golden(name)
    expect = np.array([int(r[0], 16) for r in rows], dtype=udt)
    # the definition key agrees with the hand-written order
    ranks = [definition_key(int(b), dtype) for b in expect]
    assert all(a < b for a, b in zip(ranks, ranks[1:]))
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = expect[rng.permutation(len(expect))].view(dtype)
        for out in (oracle.radix_sort(x), oracle.merge_sort(x, chunk_size=4)):
            assert np.array_equal(as_bits(out), expect)
    # the order map itself is strictly increasing along the golden list
    mapped = [oracle.ordered_bits(int(b), dtype) for b in expect]
    assert all(a < b for a, b in zip(mapped, mapped[1:]))


def test_golden_int32_example():
    rows = _read_golden("int32_example.txt")
    x = np.array([int(t) for t in rows[0]], dtype=np.int32)
    e = np.array([int(t) for t in rows[1]], dtype=np.int32)
    assert np.array_equal(oracle.radix_sort(x), e)
    assert np.array_equal(oracle.merge_sort(x, chunk_size=3), e)


# --------------------------------------------------------------------------
# Floats at size: definition via Python's stable sort with the category key.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=lambda d: np.dtype(d).name)
def test_float_specials_at_size(dtype):
    rng = np.random.default_rng(5)
    n = 20_011
    x = (rng.random(n) * 2e6 - 1e6).astype(dtype)
    x[rng.integers(0, n, 300)] = x[rng.integers(0, n, 300)]
    al = alphabet(dtype)
    pos = rng.integers(0, n, 400)
    x[pos] = al[rng.integers(0, len(al), 400)]
    v = np.arange(n, dtype=np.uint32)
    bits = as_bits(x)
    order = sorted(range(n), key=lambda i: definition_key(int(bits[i]), dtype))
    ek, ev = bits[order], np.array(order, dtype=np.uint32)
    for k, vv in (oracle.radix_sort(x, v), oracle.merge_sort(x, v, chunk_size=16)):
        assert np.array_equal(as_bits(k), ek)
        assert np.array_equal(vv, ev)
    # numpy agrees on the finite, nonzero part
    fin = x[np.isfinite(x) & (x != 0)]
    assert np.array_equal(oracle.radix_sort(fin), np.sort(fin, kind="stable"))


# --------------------------------------------------------------------------
# Invariants and special cases on generated workloads.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dist", ["uniform", "gaussian", "sorted", "reverse", "nearly_sorted",
                                  "distinct16", "zipf", "equal", "uniform1000"])
def test_invariants_on_workload_distributions(dist):
    import torch
    from paper_2505_18681_gb300 import inputs
    for tdt in (torch.int32, torch.int64):
        x = inputs.generate(dist, 3001, tdt, seed=42).numpy()
        v = np.arange(x.size, dtype=np.uint32)
        k, vv = oracle.radix_sort(x, v)
        check_invariants(x, k, v, vv)
        k2, v2 = oracle.merge_sort(x, v, chunk_size=32)
        assert np.array_equal(k, k2) and np.array_equal(vv, v2)


@pytest.mark.parametrize("dist", ["paper_uniform", "paper_normal", "paper_exponential", "paper_power",
                                  "paper_beta", "paper_sparse", "paper_clustered", "paper_nearly_sorted",
                                  "paper_duplicates"])
def test_invariants_on_paper_distributions(dist):
    import torch
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate(dist, 3001, torch.int32, seed=42).numpy()
    v = np.arange(x.size, dtype=np.uint32)
    k, vv = oracle.radix_sort(x, v)
    check_invariants(x, k, v, vv)
    assert np.array_equal(k, np.sort(x, kind="stable"))


def test_paper_distribution_shapes():
    """The paper's nine int32 distributions have the moments and structure
    their definitions fix (100,000 draws; tolerances several standard errors)."""
    import torch
    from paper_2505_18681_gb300 import inputs
    n = 100_000
    g = {d: inputs.generate(d, n, torch.int32, seed=7).numpy().astype(np.float64)
         for d in inputs.PAPER_DISTRIBUTIONS}
    for d, x in g.items():
        assert x.min() >= -1e9 and x.max() <= 1e9, d
    assert abs(g["paper_uniform"].mean()) < 1e7
    assert abs(g["paper_uniform"].std() - 2e9 / math.sqrt(12)) < 1e7
    assert abs(g["paper_normal"].mean()) < 2e6 and abs(g["paper_normal"].std() - 1e8) < 2e6
    # E[min(X, 2e9)] - 1e9 for X ~ Exp(1e9)
    assert abs(g["paper_exponential"].mean() - (1e9 * (1 - math.exp(-2)) - 1e9)) < 1e7
    assert abs(g["paper_power"].mean() - (2e9 / 3 - 1e9)) < 1e7           # E[U^2] = 1/3
    assert abs(g["paper_beta"].mean() - (2e9 * 2 / 7 - 1e9)) < 5e6         # E[Beta(2,5)] = 2/7
    assert abs((g["paper_sparse"] == 0).mean() - 0.9) < 0.01
    near = g["paper_clustered"]
    centres = -1e9 + np.arange(10) * (2e9 / 9)
    dist_to_centre = np.min(np.abs(near[:, None] - centres[None, :]), axis=1)
    assert np.mean(dist_to_centre < 3e8) > 0.99                               # 3 sigma
    ns = g["paper_nearly_sorted"]
    assert 0.88 < np.mean(ns[1:] >= ns[:-1]) < 0.93
    assert abs(len(np.unique(g["paper_duplicates"])) - n // 10) < n // 100


def test_friendster_like_shape():
    """Ids in the paper's node-id range, heavy-tailed: the most frequent id
    far above the mean count, and the most frequent ids holding the share of
    draws the rank law fixes."""
    import torch
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("friendster_like", 200_000, torch.int32, seed=42).numpy()
    assert x.min() >= 101 and x.max() <= 124_836_179
    _, counts = np.unique(x, return_counts=True)
    assert counts.max() > 50 * counts.mean()
    top = np.sort(counts)[::-1]
    # P(rank < K) = (K / M)^(1/3): the 100 lowest ranks hold about 1.15% of the
    # draws, 20 times what 100 uniformly drawn ids would
    assert top[:100].sum() > 0.008 * x.size
    k, vv = oracle.radix_sort(x, np.arange(x.size, dtype=np.uint32))
    check_invariants(x, k, np.arange(x.size, dtype=np.uint32), vv)


def test_float_mix_invariants():
    import torch
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("float_mix", 5000, torch.float64, seed=42).numpy()
    v = np.arange(x.size, dtype=np.uint32)
    k, vv = oracle.radix_sort(x, v)
    check_invariants(x, k, v, vv)


@pytest.mark.parametrize("dtype", ALL_DTYPES, ids=lambda d: np.dtype(d).name)
def test_special_cases(dtype):
    al = alphabet(dtype)
    eq = np.full(1000, al[1], dtype=dtype)
    assert np.array_equal(as_bits(oracle.radix_sort(eq)), as_bits(eq))
    s = np.sort(al[:5]) if np.dtype(dtype).kind in "iu" else al[:5]
    s = definition_sort(al)
    assert np.array_equal(as_bits(oracle.radix_sort(s)), as_bits(s))
    distinct = definition_sort(al)
    assert np.array_equal(as_bits(oracle.radix_sort(distinct[::-1].copy())), as_bits(distinct))
    assert oracle.radix_sort(np.zeros(0, dtype=dtype)).size == 0


@pytest.mark.parametrize("chunk", [1, 2, 3, 7, 32, 33, 2048, 100000])
def test_merge_chunk_sizes_agree(chunk):
    rng = np.random.default_rng(chunk)
    x = rng.integers(-50, 50, 5003).astype(np.int64)
    v = np.arange(x.size, dtype=np.uint32)
    k1, v1 = oracle.radix_sort(x, v)
    k2, v2 = oracle.merge_sort(x, v, chunk_size=chunk)
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2)


def test_segmented_definition():
    rng = np.random.default_rng(9)
    lens = rng.integers(0, 300, 60)
    lens[5] = 0
    offs = np.zeros(61, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    x = rng.integers(-2**31, 2**31, int(offs[-1]), dtype=np.int64).astype(np.int32)
    out = oracle.segmented_sort(x, offs)
    for i in range(60):
        a, b = int(offs[i]), int(offs[i + 1])
        assert np.array_equal(out[a:b], np.sort(x[a:b]))
    with pytest.raises(ValueError):
        oracle.segmented_sort(x, offs[::-1].copy())


# --------------------------------------------------------------------------
# Planted mistakes: each must be caught by a pin above.
# --------------------------------------------------------------------------
def _pins_pass():
    try:
        test_matches_numpy_stable(np.int32, 257)
        test_matches_numpy_stable(np.int64, 1000)
        test_golden_int32_example()
        test_golden_float_order("float_order_f64.txt", np.float64, np.uint64)
        test_golden_float_order("float_order_f32.txt", np.float32, np.uint32)
        test_brute_force_pairs_stability(np.int32)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("fault", [1, 2, 3, 4, 5])
def test_planted_faults_are_caught(fault):
    assert _pins_pass()
    oracle.set_fault(fault)
    try:
        assert not _pins_pass(), "fault %d slipped through the pins" % fault
    finally:
        oracle.set_fault(0)
    assert _pins_pass()


def test_segmented_generator_all_widths():
    """The segmented-workload generator covers 32- and 64-bit keys."""
    import torch
    from paper_2505_18681_gb300 import inputs
    lens = inputs.segment_lengths(50, 16, 5000, seed=1)
    for dt in (torch.int32, torch.int64, torch.uint32, torch.uint64):
        keys, offs = inputs.segmented_keys(lens, dt, seed=1)
        assert keys.numel() == int(offs[-1]) == int(lens.sum())
        out = oracle.segmented_sort(keys.numpy(), offs.numpy().astype(np.uint64))
        for i in range(0, 50, 7):
            a, b = int(offs[i]), int(offs[i + 1])
            assert np.array_equal(out[a:b], np.sort(keys.numpy()[a:b]))


# ---- the paper-shaped multithreaded CPU baseline, against the oracle ---------
@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.uint32, np.uint64, np.float32, np.float64])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_cpu_parallel_baseline_matches_oracle(dtype, threads):
    import oracle
    rng = np.random.default_rng(17)
    for n in (0, 1, 2, 7, 1000, 100_003):
        if np.dtype(dtype).kind == "f":
            x = rng.uniform(-1e6, 1e6, n).astype(dtype)
            if n > 10:
                dup = rng.integers(0, n, n // 7)
                x[dup] = x[rng.integers(0, n, dup.size)]    # duplicates
                x[3] = -0.0
                x[5] = 0.0
                x[8] = np.nan
                x[9] = -np.nan
        else:
            info = np.iinfo(dtype)
            x = rng.integers(info.min, info.max, n, dtype=dtype, endpoint=True)
            if n > 10:
                x[::5] = x[1]                                # duplicates
        got, used = oracle.parallel_radix_sort(x, threads)
        assert used == max(1, min(threads, n))
        want = oracle.radix_sort(x)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
