"""GPU parity of the batched segmented sort against the CPU oracle (each
segment sorted on its own, bit for bit), across the warp, block and large
tiers, plus offset validation and CUDA-graph capture."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def bits(a):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


@pytest.fixture(scope="module")
def evo():
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


def make(lengths, dtype, seed=42):
    from paper_2505_18681_gb300 import inputs
    lengths = torch.as_tensor(lengths, dtype=torch.int64)
    if dtype.is_floating_point:
        total = int(lengths.sum())
        keys = inputs.generate("float_mix", max(total, 1), dtype, seed=seed, device="cuda")[:total].contiguous()
        offs = torch.zeros(lengths.numel() + 1, dtype=torch.int64)
        offs[1:] = torch.cumsum(lengths, 0)
    else:
        keys, offs = inputs.segmented_keys(lengths, dtype, seed=seed, device="cuda")
    return keys, offs


def run(evo, lengths, dtype, **kw):
    keys, offs = make(lengths, dtype)
    expect = oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))
    d_offs = offs.to("cuda")
    evo.segmented_sort(keys, d_offs, **kw)
    evo.sync()
    assert np.array_equal(bits(keys), bits(expect)), "segments differ from the oracle"


TIER_LENGTHS = [0, 1, 2, 3, 31, 32, 33, 255, 256, 257, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 20_000,
                65_537, 0, 7, 150_001]


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.uint32, torch.uint64, torch.float32,
                                   torch.float64], ids=str)
def test_tier_boundaries(evo, dtype):
    run(evo, TIER_LENGTHS, dtype)


def test_log_uniform_mix_int32(evo):
    """Config-4 shape, scaled down: log-uniform lengths 16..1e5, half uniform,
    half nearly sorted segments."""
    from paper_2505_18681_gb300 import inputs
    lens = inputs.segment_lengths(3000, 16, 100_000, seed=42)
    run(evo, lens.tolist(), torch.int32)


def test_many_tiny_segments(evo):
    rng = np.random.default_rng(3)
    run(evo, rng.integers(0, 40, 20_000).tolist(), torch.int64)


@pytest.mark.parametrize("cap", [256, 1024, 4096])
def test_block_cap_param(evo, cap):
    run(evo, [100, 300, 1500, 5000, 9000, 70_000], torch.int64, seg_block_cap=cap)


def test_block_cap_sequence_in_one_process(evo):
    """Tier thresholds may change from call to call (largest last)."""
    for cap in (256, 2048, 8192):
        run(evo, [100, 3000, 7000, 9000, 40_000], torch.int32, seg_block_cap=cap)


def test_low_entropy_segments(evo):
    """Large segments whose digits are mostly constant (pass skipping inside a
    segment, including odd numbers of active passes)."""
    lens = [50_000, 70_001, 40_000, 9_999]
    for dtype in (torch.int32, torch.int64):
        keys, offs = make(lens, dtype)
        keys[: lens[0]] = 5                                    # all equal: no pass
        keys[lens[0]: lens[0] + lens[1]] %= 200                # few digits vary
        keys[lens[0] + lens[1]: lens[0] + lens[1] + lens[2]] = torch.arange(lens[2], device="cuda").to(dtype)
        expect = oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))
        evo.segmented_sort(keys, offs.to("cuda"))
        evo.sync()
        assert np.array_equal(bits(keys), bits(expect))


def test_bad_offsets_reported(evo):
    keys = torch.arange(100, dtype=torch.int32, device="cuda")
    offs = torch.tensor([0, 50, 40, 100], dtype=torch.int64, device="cuda")   # decreasing
    evo.segmented_sort(keys, offs)
    with pytest.raises(evo.EvoSortError) as ei:
        evo.sync()
    assert ei.value.status == "ERR_INVALID"
    offs = torch.tensor([0, 50, 90], dtype=torch.int64, device="cuda")        # last != total
    evo.segmented_sort(keys, offs)
    with pytest.raises(evo.EvoSortError):
        evo.sync()
    evo.sync()   # the status word is cleared after it is reported
    # a segment that ends past the array: reported, and left untouched (the
    # check skips it before any tier reads or writes its keys)
    guard = torch.arange(300, dtype=torch.int32, device="cuda").flip(0)
    keys = guard[:100]
    before = guard.clone()
    offs = torch.tensor([0, 200, 100], dtype=torch.int64, device="cuda")
    evo.segmented_sort(keys, offs)
    with pytest.raises(evo.EvoSortError) as ei:
        evo.sync()
    assert ei.value.status == "ERR_INVALID"
    assert torch.equal(guard[100:], before[100:]), "keys past the array were touched"
    evo.sync()


def test_cuda_graph_capture_and_replay(evo):
    """The whole batched sort is captured once and replayed with new keys in
    the same buffers."""
    lens = [10, 200, 3000, 9000, 40_000, 1]
    keys, offs = make(lens, torch.int32)
    d_offs = offs.to("cuda")
    work = keys.clone()
    evo.segmented_sort(work, d_offs)            # warm-up outside capture
    evo.sync()
    g = torch.cuda.CUDAGraph()
    work.copy_(keys)
    with torch.cuda.graph(g):
        evo.segmented_sort(work, d_offs)
    for seed in (1, 2):
        fresh, _ = make(lens, torch.int32, seed=seed)
        work.copy_(fresh)
        g.replay()
        torch.cuda.synchronize()
        expect = oracle.segmented_sort(fresh.cpu().numpy(), offs.numpy().astype(np.uint64))
        assert np.array_equal(bits(work), bits(expect))


@pytest.mark.parametrize("cap", [32, 64, 128, 256])
def test_warp_tier_cut_over(evo, cap):
    """Every warp-tier cut-over: lengths around each power of two go to the
    warp or the block tier; the result is the oracle's either way."""
    lengths = [0, 1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 600, 5000]
    run(evo, lengths, torch.int32, seg_warp_cap=cap)
    run(evo, lengths, torch.float64, seg_warp_cap=cap)


def test_giant_segment_takes_the_device_wide_path(evo):
    """One 5e7-key segment among 10,000 small ones: the giant segment is
    sorted by the device-wide radix path (its onesweep launches appear),
    the rest by the persistent launch; every segment matches the oracle."""
    from paper_2505_18681_gb300 import inputs
    small = inputs.segment_lengths(10_000, 16, 5_000, seed=8).tolist()
    lengths = list(small[:5000]) + [50_000_000] + list(small[5000:])
    keys, offs = make(lengths, torch.int32, seed=9)
    expect = oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))
    d_offs = offs.to("cuda")
    evo.profile(True)
    try:
        evo.segmented_sort(keys, d_offs)
        evo.sync()
        kinds = [r["kind"] for r in evo.profile_read()]
    finally:
        evo.profile(False)
    assert "radix_onesweep" in kinds and "segmented" in kinds
    assert np.array_equal(bits(keys), bits(expect))


def test_giant_tier_off_and_under_capture(evo):
    """seg_giant=-1 keeps every segment in the persistent launch; a captured
    batch (no host read possible) does the same; both match the oracle."""
    lengths = [2_000_000, 300, 70_000, 5, 1_100_000]
    run(evo, lengths, torch.int64, seg_giant=-1)
    run(evo, lengths, torch.int64, seg_giant=1 << 20)
    keys, offs = make(lengths, torch.int64, seed=4)
    expect = oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))
    d_offs = offs.to("cuda")
    work = keys.clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        evo.segmented_sort(work, d_offs, seg_giant=1 << 20, stream=s)   # warm-up outside capture
        evo.sync(s)
        g = torch.cuda.CUDAGraph()
        work.copy_(keys)
        with torch.cuda.graph(g, stream=s):
            evo.segmented_sort(work, d_offs, seg_giant=1 << 20, stream=s)
    work.copy_(keys)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(bits(work), bits(expect))


def test_segmented_table_entry_is_used(evo):
    """A tuned entry for segmented batches (class 'segmented') is taken when
    the caller leaves the choice open; the result is the oracle's."""
    evo.table_clear()
    try:
        evo.table_set(torch.int32, 20, "segmented", {"algo": 0, "seg_block_cap": 1024, "seg_warp_cap": 64,
                                                     "seg_giant": -1, "insertion_threshold": 8})
        run(evo, [10, 70, 300, 2000, 9000, 40_000, 1_000_000], torch.int32)
    finally:
        evo.table_clear()
