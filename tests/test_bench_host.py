"""Host-side parts of bench.py that need no GPU: the clock sampler (against a stand-in
nvidia-smi that prints rows in the query's CSV format), the per-box work counts, and the
guards on the DRAM traffic records."""

import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1802_00330_gb300 import synth  # noqa: E402


def _fake_smi(tmp_path, rows):
    path = tmp_path / "nvidia-smi"
    lines = "\n".join(f'echo "{r}"; sleep 0.05' for r in rows)
    path.write_text(f"#!/bin/bash\n{lines}\nwhile true; do echo \"{rows[-1]}\"; sleep 0.05; done\n")
    path.chmod(path.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_clock_sampler_brackets_a_short_region(tmp_path, monkeypatch):
    row = "0, 2070, 2070, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1980, 2070, 1400.00, 0x4, Not Active, Not Active, Not Active, Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, [row, capped, row]) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    assert len(c.rows) >= 1          # a sample is in before the region starts
    time.sleep(0.001)                # a region far shorter than the sampling period
    r = c.stop()
    assert r["samples"] >= 2
    assert r["sm_max_mhz"] == 2070.0
    assert r["sm_mhz"] in (1980.0, 2025.0, 2070.0)


def test_clock_sampler_reports_reasons(tmp_path, monkeypatch):
    capped = "0, 1980, 2070, 1400.00, 0x4, Not Active, Not Active, Not Active, Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, [capped]) + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r["reasons"] == ["sw_power_cap"] and r["sm_mhz"] == 1980.0


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    monkeypatch.setenv("PATH", "/nonexistent")
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_work_counts_of_the_n6_system():
    """Per-box FP64 operation counts the roofline uses (2306 Gauss-Seidel, 2342 Krawczyk,
    304 per evaluation for the n = 6 system)."""
    s = synth.config_n6()
    assert bench.hs_ops(s) == 2306
    assert bench.hs_ops(s, krawczyk=True) == 2342
    assert bench.eval_ops(s) == 304


def test_traffic_records_apply_only_to_their_kernel_sources_and_sweep_size(monkeypatch):
    """A DRAM traffic record is reported only for the kernel sources it was captured
    with (code hash), for default options, and at the sweep size it was taken at; a per-box
    record scales with the boxes a launch processes."""
    rec = bench.TRAFFIC[("batched", "hs_n8")]
    monkeypatch.setattr(bench, "hs_sources_sha", lambda read=None, files=bench.KERNEL_SOURCES: rec["sources_sha256"])
    w = rec["wave_children"]
    assert bench.traffic_of("batched", "hs_n8", True, 1000, w) == rec["bytes_per_hs_box"] * 1000
    assert bench.traffic_of("batched", "hs_n8", True, 1000, w // 4) is None     # another sweep size
    assert bench.traffic_of("batched", "hs_n8", False, 1000, w) is None         # non-default options
    assert bench.traffic_of("batched", "hs_n8", True, None, w) is None          # boxes per launch unknown
    assert bench.traffic_of("batched", "eval", True, 1000, w) is None           # no record
    monkeypatch.setattr(bench, "hs_sources_sha", lambda read=None, files=bench.KERNEL_SOURCES: "0" * 64)
    assert bench.traffic_of("batched", "hs_n8", True, 1000, w) is None          # kernel sources changed


def test_code_hash_ignores_comments_and_whitespace():
    a = "int f(int x) {  // a comment\n  return x + 1; /* block\n comment */ }\n"
    b = "int f(int x) {\n\treturn x + 1; }"
    c = "int f(int x) { return x + 2; }"
    src = {"a": a, "b": b, "c": c}
    ha = bench.hs_sources_sha(read=lambda f: src["a"], files=("x",))
    hb = bench.hs_sources_sha(read=lambda f: src["b"], files=("x",))
    hc = bench.hs_sources_sha(read=lambda f: src["c"], files=("x",))
    assert ha == hb and ha != hc
