"""The dispatcher's host logic (Algorithm 5, AdaptivePartitionSort), on the CPU.

`evosort_plan_host` reads a strided sample of keys in host memory, classifies
it and looks the class up in the tuned table, with no device access, so the
classification rules and the table lookup run here: each class from inputs
built to have exactly its property, the priority between classes, the key
map under the sample (float order, descending), and the lookup's fallbacks
(nearest size bucket, then the random class, then the defaults)."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def evo():
    from paper_2505_18681_gb300 import _build
    _build.build()
    import paper_2505_18681_gb300 as evo
    evo.library()
    evo.table_clear()
    yield evo
    evo.table_clear()


TAGGED = ("random", "skewed", "narrow", "few", "sorted", "reverse", "constant", "narrow16")


def tag(cls):
    """An insertion threshold that names the table entry it came from."""
    return 100 + TAGGED.index(cls)


@pytest.fixture()
def table(evo):
    """One entry per class for int64 at size bucket 20 (2^20 keys)."""
    evo.table_clear()
    for cls in TAGGED:
        evo.table_set(torch.int64, 20, cls, {"algo": 0, "insertion_threshold": tag(cls)})
    yield evo
    evo.table_clear()


def rng(seed):
    return np.random.default_rng(seed)


N = 1 << 20


def uniform64(n, seed):
    return rng(seed).integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, n, dtype=np.int64,
                              endpoint=True)


def cases():
    """(name, keys, expected class) built so exactly the named property holds."""
    r = rng(1)
    asc = np.cumsum(r.integers(1, 1000, N)).astype(np.int64) - 10 ** 8   # strictly rising, both signs
    skew = uniform64(N, 2)
    pick = r.random(N) < 0.4                     # 40% of the keys in [0, 2^40): top mapped byte 0x80
    skew[pick] = r.integers(0, 1 << 40, int(pick.sum()))
    return [
        ("constant", np.full(N, -5, np.int64), "constant"),
        ("few", r.integers(-25, 25, N).astype(np.int64), "few"),
        ("sorted", asc, "sorted"),
        ("reverse", asc[::-1].copy(), "reverse"),
        ("nearly_sorted", _swap_some(asc, 0.01, 3), "sorted"),
        ("narrow16", r.integers(0, 60000, N).astype(np.int64), "narrow16"),
        ("narrow", r.integers(0, 1 << 30, N).astype(np.int64), "narrow"),
        ("skewed", skew, "skewed"),
        ("random", uniform64(N, 4), "random"),
        # both signs near zero: the mapped keys differ in the top bit, so not narrow, and half
        # of them share the top byte 0x7F, the other half 0x80: skewed
        ("signed_small", r.integers(-30000, 30000, N).astype(np.int64), "skewed"),
    ]


def _swap_some(a, frac, seed):
    a = a.copy()
    r = rng(seed)
    i = r.integers(0, a.size, int(a.size * frac))
    j = r.integers(0, a.size, int(a.size * frac))
    a[i], a[j] = a[j], a[i]
    return a


@pytest.mark.parametrize("name,keys,want", cases(), ids=[c[0] for c in cases()])
def test_each_class_and_its_table_entry(table, name, keys, want):
    p, cls = table.plan_host(torch.from_numpy(keys))
    assert cls == want
    assert p["insertion_threshold"] == tag(want)


def test_few_values_take_priority_over_order(table):
    """At most 64 distinct sampled values reads as few, even in order."""
    keys = np.repeat(np.arange(40, dtype=np.int64), N // 40 + 1)[:N]
    assert table.plan_host(torch.from_numpy(keys))[1] == "few"
    keys = np.repeat(np.arange(100, dtype=np.int64), N // 100 + 1)[:N]
    assert table.plan_host(torch.from_numpy(keys))[1] == "sorted"


def test_order_ignores_equal_neighbours(table):
    """Long runs of equal keys between strict rises: sorted, not both."""
    keys = np.repeat(np.arange(1000, dtype=np.int64) * 7, N // 1000 + 1)[:N]
    assert table.plan_host(torch.from_numpy(keys))[1] == "sorted"


def test_descending_reads_the_sample_in_the_sort_direction(table):
    asc = np.arange(N, dtype=np.int64) * 3 - N
    assert table.plan_host(torch.from_numpy(asc), descending=True)[1] == "reverse"
    assert table.plan_host(torch.from_numpy(asc[::-1].copy()), descending=True)[1] == "sorted"


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=str)
def test_float_order_under_the_sample(evo, dtype):
    """Rising floats of both signs (raw bits fall over the negatives) read as
    sorted only through the total-order map."""
    evo.table_clear()
    evo.table_set(dtype, 20, "random", {"algo": 0})
    x = torch.linspace(-1e6, 1e6, N, dtype=torch.float64).to(dtype)
    assert torch.all(x[1:] > x[:-1])
    assert evo.plan_host(x)[1] == "sorted"
    assert evo.plan_host(x.flip(0).contiguous())[1] == "reverse"
    assert evo.plan_host(x, descending=True)[1] == "reverse"
    evo.table_clear()


def defaults(evo):
    """The library's default parameters (what a lookup without an entry returns)."""
    import ctypes
    p = evo.Params()
    evo.library().evosort_default_params(ctypes.byref(p))
    return evo.params_dict(p)


def test_lookup_fallbacks(evo):
    evo.table_clear()
    evo.table_set(torch.int64, 12, "few", {"algo": 0, "insertion_threshold": 201})
    evo.table_set(torch.int64, 24, "few", {"algo": 0, "insertion_threshold": 202})
    evo.table_set(torch.int64, 20, "random", {"algo": 0, "insertion_threshold": 203})
    few = lambda n: torch.from_numpy(rng(n).integers(0, 10, n).astype(np.int64))
    assert evo.plan_host(few(1 << 13))[0]["insertion_threshold"] == 201   # bucket 13: nearest is 12
    assert evo.plan_host(few(1 << 23))[0]["insertion_threshold"] == 202   # bucket 23: nearest is 24
    # the random class's own entry, at the nearest bucket (16 -> 20)
    p, cls = evo.plan_host(torch.from_numpy(uniform64(1 << 16, 5)))
    assert cls == "random" and p["insertion_threshold"] == 203
    # a class with no entry takes the random class's entry
    p, cls = evo.plan_host(torch.from_numpy(np.arange(1 << 16, dtype=np.int64)))
    assert cls == "sorted" and p["insertion_threshold"] == 203
    # no entry for the key type: the defaults
    p, _ = evo.plan_host(torch.from_numpy(np.arange(1 << 16, dtype=np.int32)))
    assert p == defaults(evo)
    evo.table_clear()


def test_empty_table_or_single_key_is_not_sampled(evo):
    evo.table_clear()
    p, cls = evo.plan_host(torch.from_numpy(np.full(1 << 16, 3, np.int64)))
    assert cls == "random" and p == defaults(evo)
    evo.table_set(torch.int64, 0, "constant", {"algo": 0, "insertion_threshold": 7})
    p, cls = evo.plan_host(torch.tensor([42], dtype=torch.int64))
    assert cls == "random" and p == defaults(evo)
    evo.table_clear()


@pytest.mark.parametrize("dtype", [torch.int32, torch.int64], ids=str)
def test_tuning_workloads_sample_as_their_class(evo, dtype):
    """Each class's tuning workload is read as that class by the dispatcher,
    so the entry the GA writes is the one the sample later selects.  For
    32-bit keys the narrow class cannot occur (narrow16 takes every sample
    with at most half the key bits varying); its workload reads as skewed."""
    import importlib
    from paper_2505_18681_gb300 import inputs
    tm = importlib.import_module("paper_2505_18681_gb300.tune")
    evo.table_clear()
    evo.table_set(dtype, 20, "random", {"algo": 0})
    for cls, dist in tm.REPRESENTATIVE.items():
        x = inputs.generate(dist, N, dtype, seed=42, device="cpu")
        want = "skewed" if (dtype == torch.int32 and cls == "narrow") else cls
        assert evo.plan_host(x)[1] == want, (cls, dist)
    evo.table_clear()
