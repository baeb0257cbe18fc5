"""Host-side checks of the genetic algorithm (Algorithm 2) and the tuned
table, with a synthetic fitness function instead of device timings."""
import math

import pytest


@pytest.fixture(scope="module")
def evo():
    from paper_2505_18681_gb300 import _build
    _build.build()
    import paper_2505_18681_gb300 as evo
    evo.library()
    return evo


def landscape(p, _best):
    """Synthetic sort times: radix with d=11, 512x32 tiles and ballot ranking
    is the unique optimum; mergesort is slower and prefers T_ins near 48."""
    if p["algo"] == 1:
        return 50.0 + abs(p["insertion_threshold"] - 48) * 0.1
    t = 10.0 + abs(p["digit_bits"] - 11) * 1.5
    t += 0.0 if (p["block_size"], p["keys_per_thread"]) == (512, 32) else 2.0
    t += 0.0 if p["rank_mode"] == 2 else 1.0
    return t


def test_converges_to_the_optimum(evo):
    best, ms, log = evo.ga_search(landscape, key_bytes=4, seed=7)
    assert best["algo"] == 0 and best["digit_bits"] == 11 and best["rank_mode"] == 2
    assert (best["block_size"], best["keys_per_thread"]) == (512, 32)
    assert ms == pytest.approx(10.0)
    assert len(log) == 10


def test_elitism_keeps_the_best_and_log_is_consistent(evo):
    _, ms, log = evo.ga_search(landscape, key_bytes=8, seed=3)
    bests = [g["best_ms"] for g in log]
    assert all(b2 <= b1 for b1, b2 in zip(bests, bests[1:])), bests
    for g in log:
        assert g["best_ms"] <= g["mean_ms"] <= g["worst_ms"]
    assert ms == min(bests)
    evals = [g["evaluations"] for g in log]
    assert all(e2 >= e1 for e1, e2 in zip(evals, evals[1:]))
    assert evals[-1] < 30 * 10     # identical genomes are timed once


def test_seeded_determinism(evo):
    a = evo.ga_search(landscape, key_bytes=8, seed=11, generations=6)
    b = evo.ga_search(landscape, key_bytes=8, seed=11, generations=6)
    assert a == b
    c = evo.ga_search(landscape, key_bytes=8, seed=12, generations=6)
    assert c[2] != a[2] or c[0] == a[0]


def test_failed_genomes_are_discarded(evo):
    """Genomes the fitness rejects (negative) never win."""
    def picky(p, best):
        return -1.0 if p["rank_mode"] == 2 else landscape(p, best)
    best, ms, _ = evo.ga_search(picky, key_bytes=4, seed=5)
    assert best["rank_mode"] != 2 and math.isfinite(ms)


def test_first_generation_holds_the_defaults(evo):
    seen = []

    def record(p, best):
        seen.append(p)
        return landscape(p, best)
    evo.ga_search(record, key_bytes=8, seed=1, generations=1)
    assert {"algo": 0, "digit_bits": 8, "rank_mode": 4}.items() <= seen[0].items()


def test_merge_only_when_allowed(evo):
    def merge_fast(p, best):
        return 1.0 if p["algo"] == 1 else landscape(p, best)
    best, _, _ = evo.ga_search(merge_fast, key_bytes=8, seed=2)
    assert best["algo"] == 1
    best, _, _ = evo.ga_search(merge_fast, key_bytes=8, seed=2, allow_merge=0)
    assert best["algo"] == 0


def test_bad_ga_config_rejected(evo):
    with pytest.raises(evo.EvoSortError):
        evo.ga_search(landscape, population=2)
    with pytest.raises(evo.EvoSortError):
        evo.ga_search(landscape, elite=40)


def test_table_save_load_roundtrip(evo, tmp_path):
    import torch
    evo.table_clear()
    evo.table_set(torch.int64, 29, "random", {"algo": 0, "digit_bits": 11, "block_size": 512,
                                              "keys_per_thread": 16, "rank_mode": 2}, 12.5)
    evo.table_set(torch.int64, 29, "few", {"algo": 0, "digit_bits": 8, "rank_mode": 2}, 3.0)
    evo.table_set(torch.int32, 20, "sorted", {"algo": 1, "insertion_threshold": 64}, 1.0)
    evo.table_set(torch.int64, 29, "random", {"algo": 0, "digit_bits": 10, "rank_mode": 2}, 11.0)  # replaces
    assert evo.table_size() == 3
    path = str(tmp_path / "table.txt")
    evo.table_save(path)
    evo.table_clear()
    assert evo.table_size() == 0
    evo.table_load(path)
    assert evo.table_size() == 3
    text = (tmp_path / "table.txt").read_text()
    assert "1 29 0 0 10" in text
    evo.table_clear()
    bad = tmp_path / "bad.txt"
    bad.write_text("1 29 0 zero\n")
    with pytest.raises(evo.EvoSortError):
        evo.table_load(str(bad))
    evo.table_clear()
