"""Host-side parts of bench.py that need no GPU: the clock sampler (against a stand-in
nvidia-smi that prints rows in the query's CSV format) and the per-box work counts."""

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
