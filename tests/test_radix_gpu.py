"""GPU parity of the LSD radix path (Algorithms 4a/4b) against the CPU oracle.

Every case compares the CUDA result with the oracle's bit for bit on the same
seeded input (the oracle sorts a host copy of the exact device input).  Sizes
span one tile, several tiles and ragged tails; parameters cover every digit
width, tile shape and ranking variant compiled into the library.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

INT = [torch.int32, torch.int64, torch.uint32, torch.uint64]
ALL = INT + [torch.float32, torch.float64]


def bits(t: torch.Tensor) -> np.ndarray:
    a = t.cpu().numpy()
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def gen(dist, n, dtype, seed=42):
    from paper_2505_18681_gb300 import inputs
    if dtype.is_floating_point and dist != "float_mix":
        dist = "uniform"
    return inputs.generate(dist, n, dtype, seed=seed, device="cuda")


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


def run_keys(evo, x, inplace=False, **kw):
    expect = oracle.radix_sort(x.cpu().numpy())
    if inplace:
        y = x.clone()
        evo.sort(y, **kw)
    else:
        y = torch.empty_like(x)
        x0 = x.clone()
        evo.sort(x, out=y, **kw)
    evo.sync()
    assert np.array_equal(bits(y), expect.view(bits(y).dtype)), "keys differ from the oracle"
    if not inplace:
        assert torch.equal(x.view(torch.uint8), x0.view(torch.uint8)), "input modified"


def run_pairs(evo, x, inplace=False, **kw):
    n = x.numel()
    v = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
    ek, ev = oracle.radix_sort(x.cpu().numpy(), v.cpu().numpy())
    if inplace:
        k, vv = x.clone(), v.clone()
        evo.sort_pairs(k, vv, **kw)
    else:
        k, vv = torch.empty_like(x), torch.empty_like(v)
        evo.sort_pairs(x, v, k, vv, **kw)
    evo.sync()
    assert np.array_equal(bits(k), ek.view(bits(k).dtype)), "pair keys differ"
    assert np.array_equal(vv.cpu().numpy(), ev), "pair values (stable argsort) differ"


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 255, 2048, 4095, 4096, 4097, 3 * 4096 + 17, 100_003])
def test_sizes(evo, dtype, n):
    run_keys(evo, gen("uniform", n, dtype), algo="radix")


def test_config_1e6_int32_seed0(evo):
    """1e6 int32 keys uniform over the full range, seed 0, 8-bit digits."""
    run_keys(evo, gen("uniform", 1_000_000, torch.int32, seed=0), algo="radix", digit_bits=8)
    run_keys(evo, gen("uniform", 1_000_000, torch.int32, seed=0), inplace=True, algo="radix", digit_bits=8)


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "sorted", "reverse", "nearly_sorted",
                                  "distinct16", "zipf", "equal", "uniform1000", "uniform_paper"])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_distributions(evo, dist, dtype):
    x = gen(dist, 300_007, dtype)
    run_keys(evo, x, algo="radix")
    run_keys(evo, x, inplace=True, algo="radix")
    run_pairs(evo, x, algo="radix")


@pytest.mark.parametrize("d", list(range(4, 12)))
@pytest.mark.parametrize("dtype", [torch.int32, torch.float64], ids=str)
def test_digit_widths(evo, d, dtype):
    """Every digit width; odd pass counts also exercise the in-place copy-back."""
    x = gen("float_mix" if dtype.is_floating_point else "uniform", 70_001, dtype)
    run_keys(evo, x, algo="radix", digit_bits=d)
    run_keys(evo, x, inplace=True, algo="radix", digit_bits=d)
    run_pairs(evo, x, inplace=True, algo="radix", digit_bits=d)


def tile_fits(block, kpt, w, pairs, d, rank):
    """Shared memory of one radix CTA: three tile buffers, per-warp digit
    counters (two virtual warps per warp), digit offsets, counts, partial sums
    and bases, two mbarriers (<= 227 KB less 1 KB).
    Rank mode 3 keeps its match masks in the reorder buffer."""
    return smem_vw(block, kpt, w, pairs, d, vw_of(block, kpt, w, pairs, d, rank)) <= LIMIT


LIMIT = 232448 - 1024


def smem_vw(block, kpt, w, pairs, d, vw):
    s = 3 * block * kpt * (w + (4 if pairs else 0)) + block // 32 * vw * (1 << d) * 2 + (1 << d) * 20 + 16
    if (2 << d) <= block:
        s += (1 << d) * 16
    return s


def vw_of(block, kpt, w, pairs, d, rank=0):
    """Two virtual warps per warp where their counters (and, for match-mask
    ranking, their masks in the reorder buffer) fit, else one."""
    masks_ok = rank not in (3, 4) or block // 32 * 2 * (1 << d) * 4 <= block * kpt * w
    return 2 if kpt % 2 == 0 and smem_vw(block, kpt, w, pairs, d, 2) <= LIMIT and masks_ok else 1


@pytest.mark.parametrize("shape", [(256, 8), (256, 16), (1024, 4), (512, 8), (512, 16), (512, 32), (1024, 8),
                                   (1024, 16)])
@pytest.mark.parametrize("rank", [1, 2, 3, 4])
@pytest.mark.parametrize("d", [6, 8, 11])
def test_tile_shapes_and_ranking(evo, shape, rank, d):
    """Every compiled staged-tile shape and ranking variant; shapes whose tile
    does not fit in shared memory, match.any ranking at a width other than 8
    bits and match-mask ranking above 8 bits must be rejected with ERR_INVALID."""
    block, kpt = shape
    kw = dict(algo="radix", block_size=block, keys_per_thread=kpt, rank_mode=rank, digit_bits=d, pass_kernel=1)
    for dtype in (torch.uint32, torch.int64):
        w = 4 if dtype == torch.uint32 else 8
        x = gen("zipf" if dtype == torch.int64 else "uniform", 150_011, dtype)
        for pairs in (False, True):
            runner = run_pairs if pairs else run_keys
            compiled = rank == 2 or (rank in (1, 4) and d == 8) or (rank == 3 and d <= 8)
            masks_fit = rank not in (3, 4) or \
                block // 32 * vw_of(block, kpt, w, pairs, d, 3) * (1 << d) * 4 <= block * kpt * w
            if compiled and masks_fit and tile_fits(block, kpt, w, pairs, d, rank):
                runner(evo, x, **kw)
            else:
                with pytest.raises(evo.EvoSortError) as ei:
                    runner(evo, x, **kw)
                assert ei.value.status == "ERR_INVALID"


REG_SHAPES = {(4, False): [(1024, 16), (512, 16)], (4, True): [(1024, 12), (1024, 8)],
              (8, False): [(1024, 12), (1024, 8), (512, 8)], (8, True): [(1024, 12), (1024, 8), (512, 8)]}


@pytest.mark.parametrize("dtype", ALL, ids=str)
@pytest.mark.parametrize("pairs", [False, True], ids=["keys", "pairs"])
def test_register_tile_shapes(evo, dtype, pairs):
    """Every compiled register-tile shape (pass_kernel 2) with match masks,
    match.any and adaptive ranking, at sizes around one tile, several tiles
    with a ragged tail, in place and out of place, against the oracle."""
    w = torch.empty(0, dtype=dtype).element_size()
    runner = run_pairs if pairs else run_keys
    for block, kpt in REG_SHAPES[(w, pairs)]:
        tile = block * kpt
        for n in (1, tile - 1, tile + 1, 5 * tile + 37):
            x = gen("float_mix" if dtype.is_floating_point else "gaussian", n, dtype, seed=n % 97)
            for rank in (1, 3, 4):
                runner(evo, x, algo="radix", pass_kernel=2, block_size=block, keys_per_thread=kpt, rank_mode=rank)
            runner(evo, x, inplace=True, algo="radix", pass_kernel=2, block_size=block, keys_per_thread=kpt)


def test_register_tile_rejections(evo):
    """The register tile exists for 8-bit digits and rank modes 1, 3 and 4:
    other requests for it are rejected, and pass_kernel outside 0..2 too."""
    x = gen("uniform", 10_000, torch.int32)
    for kw in (dict(digit_bits=6), dict(rank_mode=2), dict(block_size=256, keys_per_thread=8)):
        with pytest.raises(evo.EvoSortError) as ei:
            run_keys(evo, x, algo="radix", pass_kernel=2, **kw)
        assert ei.value.status == "ERR_INVALID"
    with pytest.raises(evo.EvoSortError) as ei:
        run_keys(evo, x, algo="radix", pass_kernel=3)
    assert ei.value.status == "ERR_INVALID"


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "distinct16", "sorted"])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_staged_and_register_tiles_agree_with_oracle(evo, dist, dtype):
    """Both pass kernels at their default shapes on the same input, each
    against the oracle (the default picks the register tile)."""
    x = gen(dist, ADAPT_N, dtype, seed=21)
    run_keys(evo, x, algo="radix", pass_kernel=1)
    run_keys(evo, x, algo="radix", pass_kernel=2)
    run_pairs(evo, x, algo="radix", pass_kernel=1)
    run_pairs(evo, x, algo="radix", pass_kernel=2)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=str)
def test_float_total_order_and_stability(evo, dtype):
    """-0.0 < +0.0, NaNs last with payloads kept, stable argsort (config 3 shape)."""
    x = gen("float_mix", 200_003, dtype)
    run_keys(evo, x, algo="radix")
    run_pairs(evo, x, algo="radix")
    run_pairs(evo, x, inplace=True, algo="radix")


def test_unaligned_and_offset_views(evo):
    """Keys that start off a 16-byte boundary (histogram head/tail path)."""
    for dtype in (torch.int32, torch.int64):
        base = gen("uniform", 50_013, dtype)
        for off in (1, 2, 3):
            x = base[off:].contiguous() if off == 0 else base[off:]
            run_keys(evo, x, algo="radix")


def test_all_passes_skipped(evo):
    """All-equal keys: every digit is constant, no pass runs; out-of-place
    copies, in-place is a no-op; values keep input order."""
    for dtype in ALL:
        x = torch.full((12_345,), 7, dtype=torch.int64, device="cuda").to(dtype) if not dtype.is_floating_point \
            else torch.full((12_345,), -0.0, dtype=dtype, device="cuda")
        run_keys(evo, x, algo="radix")
        run_keys(evo, x, inplace=True, algo="radix")
        run_pairs(evo, x, algo="radix")


def test_caller_workspace_and_stream(evo):
    x = gen("uniform", 123_457, torch.int64)
    need = evo.workspace_bytes(x.numel(), torch.int64, with_values=False, algo="radix")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        evo.sort(x, out=y, algo="radix", workspace=ws)
    evo.sync(s)
    assert np.array_equal(bits(y), oracle.radix_sort(x.cpu().numpy()).view(np.uint64))
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(evo.EvoSortError) as ei:
        evo.sort(x, out=y, algo="radix", workspace=small)
    assert ei.value.status == "ERR_NOMEM"


def test_repeated_calls_are_identical(evo):
    x = gen("gaussian", 500_001, torch.int64)
    outs = []
    for _ in range(3):
        y = torch.empty_like(x)
        evo.sort(x, out=y, algo="radix", digit_bits=11)
        outs.append(y)
    evo.sync()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])


@pytest.mark.parametrize("dist", ["sorted", "equal", "distinct16", "uniform1000"])
def test_match_mask_ranking_low_entropy(evo, dist):
    """Rank mode 3 when whole warps share a digit (its slow case) is still exact."""
    for dtype in (torch.int32, torch.int64):
        x = gen(dist, 200_003, dtype)
        run_pairs(evo, x, algo="radix", rank_mode=3, digit_bits=8)
        run_keys(evo, x, algo="radix", rank_mode=3, digit_bits=5)


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "distinct16"])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_many_tiles_per_cta(evo, dist, dtype):
    """Enough tiles that every persistent CTA runs many iterations and the
    look-back walks over tiles of every state (published aggregate,
    inclusive prefix, not yet published)."""
    run_keys(evo, gen(dist, 12_000_017, dtype, seed=5))


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float64], ids=str)
def test_digit_prefix_above_2_24(evo, dtype):
    """One digit held by 90% of 20M keys in every pass: per-digit inclusive
    prefixes in the 32-bit look-back slots pass 2^24 (all passes stay active
    through the other 10%)."""
    n = 20_000_000
    x = gen("uniform", n, dtype, seed=11)
    pick = gen("uniform", n, torch.int64, seed=12).remainder(10) != 0
    x = torch.where(pick, torch.full_like(x, 3), x)
    run_keys(evo, x)


ADAPT_N = 3_000_017   # above the size where adaptive ranking starts (2^21 keys)


@pytest.mark.parametrize("dist", ["gaussian", "distinct16", "zipf", "uniform1000", "sorted", "uniform"])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float64], ids=str)
def test_adaptive_ranking(evo, dist, dtype):
    """Rank mode 4 (the default): every pass launches the match-mask and the
    match.any kernel and exactly one of them runs; the result is the oracle's,
    for keys and for stable pairs."""
    x = gen(dist, ADAPT_N, dtype, seed=9)
    evo.profile(True)
    try:
        run_keys(evo, x, algo="radix", rank_mode=4, digit_bits=8)
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep"]
    finally:
        evo.profile(False)
    passes = {}
    for r in recs:
        passes.setdefault(r["pass"], []).append(r)
    assert len(passes) == 8 * x.element_size() // 8
    for p, rs in passes.items():
        assert sorted(r["rank"] for r in rs) == [1, 3]
        assert sum(r["active"] for r in rs) <= 1
    run_pairs(evo, x, algo="radix", rank_mode=4, digit_bits=8)


def test_adaptive_ranking_choice_per_pass(evo):
    """Gaussian int64 keys (sd 1e6) with a few keys at both ends of the int64
    range (so the span needs all eight digits and the sort is not rebased):
    the five top bytes take two values for nearly every key, so passes 3..7
    run match.any; passes 0..2 (spread digits, the first pass in input order)
    run match masks."""
    x = gen("gaussian", ADAPT_N, torch.int64, seed=9)
    x[::1_000_003] = torch.iinfo(torch.int64).min + 5
    x[7::1_000_003] = torch.iinfo(torch.int64).max - 5
    y = torch.empty_like(x)
    evo.profile(True)
    try:
        evo.sort(x, out=y, algo="radix", rank_mode=4, digit_bits=8)
        evo.sync()
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep" and r["active"]]
    finally:
        evo.profile(False)
    assert {r["pass"]: r["rank"] for r in recs} == {0: 3, 1: 3, 2: 3, 3: 1, 4: 1, 5: 1, 6: 1, 7: 1}
    assert np.array_equal(bits(y), oracle.radix_sort(x.cpu().numpy()).view(np.uint64))


def test_below_adaptive_size_single_launch_per_pass(evo):
    x = gen("gaussian", 100_003, torch.int64)
    evo.profile(True)
    try:
        run_keys(evo, x, algo="radix", rank_mode=4, digit_bits=8)
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep"]
    finally:
        evo.profile(False)
    assert len(recs) == 8 and all(r["rank"] == 0 for r in recs)


PAPER_DISTS = ["paper_uniform", "paper_normal", "paper_exponential", "paper_power", "paper_beta",
               "paper_sparse", "paper_clustered", "paper_nearly_sorted", "paper_duplicates", "friendster_like"]


@pytest.mark.parametrize("dist", PAPER_DISTS)
def test_paper_distributions_int32(evo, dist):
    """The paper's nine int32 distributions, through the dispatcher's choice
    with the tuned int32 table and through the defaults, keys and pairs."""
    import os
    x = gen(dist, ADAPT_N, torch.int32, seed=3)
    run_keys(evo, x, algo="radix")
    run_pairs(evo, x, algo="radix")
    table = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2505_18681_gb300",
                         "tuned", "gb300_int32.txt")
    evo.table_clear()
    evo.table_load(table)
    try:
        run_keys(evo, x)
    finally:
        evo.table_clear()


@pytest.mark.parametrize("algo", ["radix", "merge"])
def test_cuda_graph_capture_of_a_device_wide_sort(evo, algo):
    """A whole sort (histogram, plan, passes, fixup, stream-ordered scratch)
    is captured once and replayed on new keys in the same buffers."""
    n = 2_500_003
    x = gen("uniform", n, torch.int64, seed=1)
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        evo.sort(x, out=y, algo=algo, stream=s)     # warm-up outside capture (device set-up)
        evo.sync(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            evo.sort(x, out=y, algo=algo, stream=s)
    for seed in (2, 3):
        x.copy_(gen("gaussian", n, torch.int64, seed=seed))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(bits(y), oracle.radix_sort(x.cpu().numpy()).view(np.uint64))


@pytest.mark.parametrize("pass_kernel", [1, 2])
def test_lookback_wait_times_out_and_recovers(evo, pass_kernel):
    """With the look-back poll limit cut to one poll, a multi-tile sort's
    waits run out: the kernels return, evosort_sync reports ERR_TIMEOUT, and
    the next sort with the default limit matches the oracle (the context
    stays usable).  No wait is left unbounded: every other wait keeps its
    limit, and the per-digit range check keeps stores inside the array."""
    x = gen("uniform", 12_000_017, torch.int32, seed=5)
    y = torch.empty_like(x)
    evo.sync()
    evo.set_wait_limit(1)
    try:
        evo.sort(x, out=y, algo="radix", pass_kernel=pass_kernel, rank_mode=3)
        with pytest.raises(evo.EvoSortError) as ei:
            evo.sync()
        assert ei.value.status == "ERR_TIMEOUT"
    finally:
        evo.set_wait_limit(0)
    evo.sync()   # the status word was cleared when it was reported
    run_keys(evo, x, algo="radix", pass_kernel=pass_kernel)


def test_adaptive_thresholds_are_parameters(evo):
    """adapt_later=10 (1/1024) sends every pass after the first that runs to
    match.any; adapt_first=1 (1/2) keeps the first on match masks; the result
    is the oracle's."""
    x = gen("uniform", ADAPT_N, torch.int64, seed=9)
    y = torch.empty_like(x)
    evo.profile(True)
    try:
        evo.sort(x, out=y, algo="radix", rank_mode=4, adapt_later=10, adapt_first=1)
        evo.sync()
        recs = [r for r in evo.profile_read() if r["kind"] == "radix_onesweep" and r["active"]]
    finally:
        evo.profile(False)
    assert {r["pass"]: r["rank"] for r in recs} == {0: 3, 1: 1, 2: 1, 3: 1, 4: 1, 5: 1, 6: 1, 7: 1}
    assert np.array_equal(bits(y), oracle.radix_sort(x.cpu().numpy()).view(np.uint64))


def _onesweep_and_fixup(evo, fn):
    evo.profile(True)
    try:
        fn()
        evo.sync()
        recs = evo.profile_read()
    finally:
        evo.profile(False)
    active = [r for r in recs if r["kind"] == "radix_onesweep" and r["active"]]
    fix = [r for r in recs if r["kind"] == "radix_fixup" and r["active"]]
    return active, fix


@pytest.mark.parametrize("dtype", ALL, ids=str)
def test_presorted_input_is_copied(evo, dtype):
    """Input already in order (ascending, or descending for a descending
    sort): no pass runs; out of place it is copied, in place nothing moves;
    keys and stable pairs match the oracle."""
    n = 1_234_567
    x = gen("float_mix" if dtype.is_floating_point else "uniform", n, dtype, seed=3)
    srt = torch.from_numpy(oracle.radix_sort(x.cpu().numpy())).cuda()
    y = torch.empty_like(srt)
    active, fix = _onesweep_and_fixup(evo, lambda: evo.sort(srt, out=y, algo="radix"))
    assert not active and len(fix) == 1
    assert torch.equal(y.view(torch.uint8), srt.view(torch.uint8))
    z = srt.clone()
    active, fix = _onesweep_and_fixup(evo, lambda: evo.sort(z, algo="radix"))
    assert not active and not fix and torch.equal(z.view(torch.uint8), srt.view(torch.uint8))
    run_pairs(evo, srt, algo="radix")
    # a descending sort of descending keys is the same shortcut
    sint = torch.int32 if dtype.itemsize == 4 else torch.int64
    dsc = srt.view(sint).flip(0).contiguous().view(dtype)
    d = torch.empty_like(dsc)
    active, _ = _onesweep_and_fixup(evo, lambda: evo.sort(dsc, out=d, algo="radix", descending=True))
    assert not active and torch.equal(d.view(torch.uint8), dsc.view(torch.uint8))


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float64], ids=str)
def test_reversed_input_is_reversed(evo, dtype):
    """Strictly decreasing input: one reversed copy (keys and pairs, in and
    out of place).  Non-increasing input with equal neighbours: keys take the
    reversal; pairs take the passes (a reversal would swap equal keys'
    values)."""
    n = 2_000_003
    base = gen("float_mix" if dtype.is_floating_point else "uniform", n, dtype, seed=4)
    asc = torch.from_numpy(oracle.radix_sort(base.cpu().numpy())).cuda()
    # strictly decreasing: drop duplicates
    u = torch.unique_consecutive(asc.view(torch.int32 if dtype.itemsize == 4 else torch.int64))
    strict = u.flip(0).contiguous().view(dtype)
    y = torch.empty_like(strict)
    active, fix = _onesweep_and_fixup(evo, lambda: evo.sort(strict, out=y, algo="radix"))
    assert not active and len(fix) == 1
    run_keys(evo, strict, algo="radix")
    run_keys(evo, strict, inplace=True, algo="radix")
    run_pairs(evo, strict, algo="radix")
    run_pairs(evo, strict, inplace=True, algo="radix")
    # with equal neighbours
    dup = torch.repeat_interleave(strict[:300_000], 3)
    active, _ = _onesweep_and_fixup(evo, lambda: evo.sort(dup, out=torch.empty_like(dup), algo="radix"))
    assert not active
    run_keys(evo, dup, algo="radix")
    v = torch.arange(dup.numel(), dtype=torch.int64, device="cuda").to(torch.int32).view(torch.uint32)
    active, _ = _onesweep_and_fixup(evo, lambda: evo.sort_pairs(dup, v, torch.empty_like(dup), torch.empty_like(v),
                                                                algo="radix"))
    assert active, "pairs with equal keys must not take the reversal"
    run_pairs(evo, dup, algo="radix")


def test_one_pair_out_of_order_takes_the_passes(evo):
    """Sorted input with one swapped neighbour pair (at a chunk boundary and
    in the middle of a vector): the order check sees it, the passes run."""
    n = 3_000_000
    base = torch.arange(n, dtype=torch.int64, device="cuda") * 7 - 5
    for i in (512 * 16 - 1, 1_500_001, n - 2, 0):
        x = base.clone()
        x[i], x[i + 1] = base[i + 1], base[i]
        active, _ = _onesweep_and_fixup(evo, lambda: evo.sort(x, out=torch.empty_like(x), algo="radix"))
        assert active, i
        run_keys(evo, x, algo="radix")
        x32 = x.to(torch.int32)
        run_keys(evo, x32, algo="radix")
