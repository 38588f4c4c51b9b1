"""bench.py's clock sampler, on CPU with a stand-in for nvidia-smi: only the samples taken
from the start of the timed region count, the throttle reasons the driver rejects are
reported by name, and a missing nvidia-smi is reported rather than raised."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
pytest.importorskip("torch")
import bench  # noqa: E402

ROW = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"


def _fake_smi(tmp_path, rows, interval=0.05):
    """A script that prints `rows` one by one, `interval` seconds apart, then sleeps."""
    body = ["#!/bin/bash"]
    for r in rows:
        body += [f'echo "{r}"', f"sleep {interval}"]
    body += ["sleep 5"]
    p = tmp_path / "nvidia-smi"
    p.write_text("\n".join(body) + "\n")
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_samples_from_mark_on(tmp_path, monkeypatch):
    # idle clocks before the timed region, load clocks (with the power cap active) after
    rows = [ROW.format(sm=345, cap="Not Active")] * 2 + [ROW.format(sm=2070, cap="Active")] * 40
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.12)          # the idle rows are out before the timed region starts
    c.mark()
    time.sleep(0.3)
    r = c.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] >= 3


def test_short_region_waits_for_one_sample(tmp_path, monkeypatch):
    rows = [ROW.format(sm=1980, cap="Not Active")] * 40
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows, interval=0.2) + os.pathsep + os.environ["PATH"])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    c.mark()                  # a region far shorter than the sampling interval
    r = c.stop()
    assert r["samples"] >= 1 and r["sm_mhz"] == 1980.0 and r["reasons"] == []


def test_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    c = bench.Clocks(0)
    c.start()
    c.mark()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
