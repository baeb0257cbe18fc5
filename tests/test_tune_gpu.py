"""GPU checks of the dispatcher (Algorithm 5) and the GA tuner (Algorithm 2)."""
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
    yield evo
    evo.table_clear()


EXPECTED_CLASS = {"uniform": "random", "gaussian": "skewed", "sorted": "sorted", "reverse": "reverse",
                  "nearly_sorted": "sorted", "distinct16": "few", "zipf": "narrow", "equal": "constant",
                  "uniform1000": "narrow16"}


@pytest.mark.parametrize("dist", list(EXPECTED_CLASS))
def test_classify_workload_distributions(evo, dist):
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate(dist, 1_000_003, torch.int64, seed=42, device="cuda")
    assert evo.classify(x) == EXPECTED_CLASS[dist]


def test_classify_equal_neighbours_and_order(evo):
    """Equal neighbours do not count as order: 90% zeros is skewed, not
    sorted or reverse; sorted keys with many repeats are still sorted; few
    distinct values are 'few' in any order."""
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("paper_sparse", 1_000_003, torch.int32, seed=42, device="cuda")
    assert evo.classify(x) == "skewed"
    rep = torch.arange(1_000_003, device="cuda", dtype=torch.int64) // 7
    assert evo.classify(rep) == "sorted"
    assert evo.classify(rep.flip(0).contiguous()) == "reverse"
    few = inputs.generate("distinct16", 1_000_003, torch.int64, seed=42, device="cuda")
    assert evo.classify(torch.sort(few).values) == "few"


def test_tune_small_sample_against_oracle(evo):
    """The GA with the oracle's sorted sample as the reference: every winning
    genome produced the exact answer; the log is consistent."""
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("gaussian", 1 << 20, torch.int64, seed=42, device="cuda")
    expected = torch.from_numpy(oracle.radix_sort(x.cpu().numpy())).cuda()
    best, ms, log = evo.tune(x, expected=expected, population=12, generations=4, reps=2, seed=1)
    assert np.isfinite(ms) and ms > 0
    bests = [g["best_ms"] for g in log]
    assert all(b2 <= b1 + 1e-6 for b1, b2 in zip(bests, bests[1:]))
    y = torch.empty_like(x)
    evo.sort(x, out=y, **best)
    evo.sync()
    assert torch.equal(y, expected)


def test_tune_without_reference_uses_device_checks(evo):
    from paper_2505_18681_gb300 import inputs
    x = inputs.generate("distinct16", 1 << 19, torch.int32, seed=3, device="cuda")
    best, ms, _ = evo.tune(x, population=8, generations=2, reps=1, seed=2)
    y = torch.empty_like(x)
    evo.sort(x, out=y, **best)
    evo.sync()
    assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy()))


def test_dispatcher_uses_table(evo):
    from paper_2505_18681_gb300 import inputs
    evo.table_clear()
    evo.table_set(torch.int64, 19, "few", {"algo": 0, "digit_bits": 6, "block_size": 256,
                                          "keys_per_thread": 16, "rank_mode": 2})
    evo.table_set(torch.int64, 19, "random", {"algo": 1, "insertion_threshold": 24})
    x = inputs.generate("distinct16", 700_001, torch.int64, seed=5, device="cuda")
    p, cls = evo.plan(x)
    assert cls == "few" and p["digit_bits"] == 6 and p["rank_mode"] == 2
    u = inputs.generate("uniform", 600_001, torch.int64, seed=5, device="cuda")
    p, cls = evo.plan(u)
    assert cls == "random" and p["algo"] == 1 and p["insertion_threshold"] == 24
    s = inputs.generate("sorted", 500_001, torch.int64, seed=5, device="cuda")
    p, cls = evo.plan(s)                       # no "sorted" entry: falls back to "random"
    assert cls == "sorted" and p["algo"] == 1
    for t in (x, u, s):
        y = torch.empty_like(t)
        evo.sort(t, out=y)                    # params=None -> dispatcher
        z = t.clone()
        evo.sort(z, algo="auto")              # in place, algo auto
        evo.sync()
        e = oracle.radix_sort(t.cpu().numpy())
        assert np.array_equal(y.cpu().numpy(), e) and np.array_equal(z.cpu().numpy(), e)
    evo.table_clear()
    p, cls = evo.plan(x)                      # empty table: defaults, no sampling
    assert p["algo"] == 0 and p["digit_bits"] == 0


TUNED = ["gb300_int32.txt", "gb300_int64.txt"]


def table_lines(name):
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2505_18681_gb300",
                        "tuned", name)
    out = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            out.append([float(t) if "." in t else int(t) for t in line.split()])
    return out


def line_params(f):
    names = ["algo", "digit_bits", "block_size", "keys_per_thread", "rank_mode", "insertion_threshold",
             "seg_block_cap"]
    p = dict(zip(names, f[3:10]))
    extra = ["pass_kernel", "adapt_later", "adapt_first", "seg_warp_cap", "small_cap", "seg_giant"]
    p.update(zip(extra, f[11:17]))
    return p


@pytest.mark.parametrize("name", TUNED)
def test_every_tuned_table_line_matches_the_oracle(evo, name):
    """Each committed table entry, run with exactly its parameters on its
    class's representative workload (the workload it was tuned on, at a size
    the oracle sorts quickly), gives the oracle's answer bit for bit; the
    segmented entry runs on a batch of the tuned shape."""
    from paper_2505_18681_gb300 import inputs
    from paper_2505_18681_gb300.tune import REPRESENTATIVE
    classes = {v: k for k, v in evo.CLASSES.items()}
    dtype = torch.int32 if "int32" in name else torch.int64
    lines = table_lines(name)
    assert lines, name
    for f in lines:
        cls = evo.CLASSES[f[2]]
        p = line_params(f)
        if cls == "segmented":
            lens = inputs.segment_lengths(2_000, 16, 100_000, seed=6)
            keys, offs = inputs.segmented_keys(lens, dtype, seed=6, device="cuda")
            expect = oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))
            evo.segmented_sort(keys, offs.to("cuda"), **p)
            evo.sync()
            assert np.array_equal(keys.cpu().numpy(), expect), (name, f)
            continue
        assert cls in classes
        for n in (1 << 20, 3_000_017):
            x = inputs.generate(REPRESENTATIVE[cls], n, dtype, seed=42, device="cuda")
            y = torch.empty_like(x)
            evo.sort(x, out=y, **p)
            evo.sync()
            assert np.array_equal(y.cpu().numpy(), oracle.radix_sort(x.cpu().numpy())), (name, f, n)


def test_segmented_tuning_against_the_oracle(evo):
    """The GA in its segmented mode (tier cut-overs and the block tier's
    insertion threshold) with a device-timed fitness whose every candidate
    is checked against the oracle's per-segment sort."""
    from paper_2505_18681_gb300 import inputs
    lens = inputs.segment_lengths(3_000, 16, 60_000, seed=3)
    keys, offs = inputs.segmented_keys(lens, torch.int32, seed=3, device="cuda")
    expect = torch.from_numpy(oracle.segmented_sort(keys.cpu().numpy(), offs.numpy().astype(np.uint64))).cuda()
    d_offs = offs.to("cuda")
    work = torch.empty_like(keys)
    seen = []

    def fitness(p, _best):
        work.copy_(keys)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        try:
            evo.segmented_sort(work, d_offs, params=evo.make_params(**p))
        except evo.EvoSortError:
            return -1.0
        e1.record(s)
        evo.sync()
        seen.append(p)
        return e0.elapsed_time(e1) if torch.equal(work, expect) else -1.0

    best, ms, log = evo.ga_search(fitness, key_bytes=4, mode=1, population=10, generations=3, seed=4)
    assert np.isfinite(ms) and ms > 0 and len(log) == 3
    assert len({(q["seg_block_cap"], q["seg_warp_cap"], q["seg_giant"]) for q in seen}) > 1
    work.copy_(keys)
    evo.segmented_sort(work, d_offs, params=evo.make_params(**best))
    evo.sync()
    assert torch.equal(work, expect)
