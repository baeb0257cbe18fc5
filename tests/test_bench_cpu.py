"""The benchmark's measurement arithmetic, on the CPU: the roofline over a
timed region's launch records, the DRAM traffic figure taken from a committed
ncu summary only while the kernel source it was taken on is unchanged, the
clock samples' median and throttle reasons, the peak's source, and the
algorithmic bytes of a batched segmented sort."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def rec(kind, ms, nbytes, items, active=1):
    return {"kind": kind, "ms": ms, "bytes": nbytes, "items": items, "active": active, "pass": 0}


def test_roofline_counts_active_onesweep_launches_only(monkeypatch):
    monkeypatch.setattr(bench, "traffic_per_key_pass", lambda w: None)
    recs = [rec("radix_histogram", 5.0, 8e9, 1e9),
            rec("radix_onesweep", 4.0, 16e9, 1e9), rec("radix_onesweep", 6.0, 16e9, 1e9),
            rec("radix_onesweep", 0.01, 0.0, 1e9, active=0),   # a skipped pass
            rec("radix_fixup", 1.0, 16e9, 1e9)]
    r = bench.onesweep_roofline(recs, 8, 6000.0, "measured")
    assert r["achieved"] == pytest.approx(32e9 / 1e9 / 10e-3)        # 3200 GB/s
    assert r["frac"] == pytest.approx(3200.0 / 6000.0)
    assert r["active_launches"] == 2 and r["avg_active_launch_ms"] == pytest.approx(5.0)
    assert r["algorithmic_bytes_per_launch"] == 16e9
    assert r["traffic"] is None and r["bound"] == "hbm" and r["unit"] == "GB/s"
    monkeypatch.setattr(bench, "traffic_per_key_pass", lambda w: 15.0)
    assert bench.onesweep_roofline(recs, 8, 6000.0, "measured")["traffic"] == pytest.approx(15e9)
    empty = bench.onesweep_roofline([rec("radix_histogram", 1.0, 1.0, 1)], 8, 6000.0, "measured")
    assert empty["achieved"] == 0.0 and empty["active_launches"] == 0 and empty["traffic"] is None


def _fake_tree(tmp_path, w, figure, sha):
    """A copy of the kernel sources and one profile summary under tmp_path."""
    src = tmp_path / "paper_2505_18681_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("onesweep_reg.cuh", "radix.cuh", "common.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_2505_18681_gb300", "csrc", f), src / f)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / ("radix_onesweep_reg_int%d.txt" % (8 * w))).write_text(
        "# summary\n# a = comment, not a value\ndram_bytes_per_key_per_pass=%s\nkernel_sha256=%s\n" % (figure, sha))
    return src


def test_traffic_only_while_the_kernel_is_unchanged(tmp_path, monkeypatch):
    h = bench.kernel_hash()
    src = _fake_tree(tmp_path, 8, "14.5", h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_hash() == h
    assert bench.traffic_per_key_pass(8) == pytest.approx(14.5)
    assert bench.traffic_per_key_pass(4) is None                  # no summary for this width
    with open(src / "radix.cuh", "a") as f:                        # the kernel changes
        f.write("\n// edited\n")
    assert bench.kernel_hash() != h
    assert bench.traffic_per_key_pass(8) is None


def test_traffic_rejects_a_malformed_figure(tmp_path, monkeypatch):
    _fake_tree(tmp_path, 4, "n/a", bench.kernel_hash())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_key_pass(4) is None


@pytest.mark.parametrize("w", [4, 8])
def test_committed_summaries_are_current_or_withheld(w):
    """A committed summary either matches the kernel source (and its figure
    is DRAM bytes per key per pass near the algorithmic 2w) or is withheld."""
    t = bench.traffic_per_key_pass(w)
    path = os.path.join(ROOT, "profiles", "radix_onesweep_reg_int%d.txt" % (8 * w))
    text = open(path).read()
    if "kernel_sha256=%s" % bench.kernel_hash() in text:
        assert t is not None and 0.8 * 2 * w <= t <= 1.1 * 2 * w
    else:
        assert t is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_and_reasons():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
    s.proc = _Proc()
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = s.stop()
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    s.lines.append("0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Active, Not Active")
    assert s.stop()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_peak_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6789.6, "bf16_tflops": 1900}')
    assert bench.measured_peaks() == (6789.6, "measured")


def test_kernel_shares_sum_to_one():
    sh = bench.kernel_shares([rec("a", 3.0, 0, 0), rec("b", 1.0, 0, 0), rec("a", 4.0, 0, 0)])
    assert sh == {"a": 0.875, "b": 0.125}


def test_segmented_roofline_bytes_and_block_cap(tmp_path):
    # segments one CTA sorts on chip move 2w per key; longer ones w + P * 2w with P = w 8-bit passes
    assert bench.segmented_alg_bytes([10, 100, 5000], 4, 4096) == 2 * 4 * 110 + (4 + 4 * 8) * 5000
    assert bench.segmented_alg_bytes([4096, 4097], 8, 4096) == 2 * 8 * 4096 + (8 + 8 * 16) * 4097
    t = tmp_path / "table.txt"
    t.write_text("# header\n"
                 "0 20 8 0 0 0 0 0 0 2048 1.0\n"
                 "0 26 8 0 0 0 0 0 0 16384 1.0\n"
                 "1 26 8 0 0 0 0 0 0 1024 1.0\n"
                 "0 26 0 0 8 0 0 0 0 999 1.0\n")
    assert bench.segmented_block_cap(str(t), 4, 1 << 21) == 2048      # bucket 21: nearest 20
    assert bench.segmented_block_cap(str(t), 4, 1 << 25) == 16384     # bucket 25: nearest 26
    assert bench.segmented_block_cap(str(t), 8, 1 << 25) == 1024
    (tmp_path / "none.txt").write_text("0 20 0 0 8 0 0 0 0 0 1.0\n")  # no segmented entry
    assert bench.segmented_block_cap(str(tmp_path / "none.txt"), 4, 1 << 20) == 8192
    assert bench.segmented_block_cap(str(tmp_path / "none.txt"), 8, 1 << 20) == 4096


def test_reference_line_carries_the_contract_keys(monkeypatch, capsys):
    """The reference arm's JSON line (the oracle on a bounded sample) has
    every key of the benchmark line, with the metric and units of the GPU arm
    and e2e moving no bytes between host and device."""
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), {"dists": "uniform,gaussian", "cpu_sample": 2000, "warmup": 1, "steps": 2,
                          "dtype": "int64", "gpus": 1})()
    bench.reference_arm(args)
    line = json.loads(capsys.readouterr().out.strip())
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GKeys/s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    e = line["e2e"]
    assert e["value"] == line["value"] and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
