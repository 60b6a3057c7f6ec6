"""Host-side logic of bench.py on CPU: the clock sampler (against a fake
nvidia-smi that streams rows like `nvidia-smi --query-gpu=... -lms`) and the
traffic figure tied to the rollout kernel's sources."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def fake_smi(tmp_path, row):
    p = tmp_path / "nvidia-smi"
    p.write_text("#!/bin/bash\nwhile true; do echo \"%s\"; sleep 0.02; done\n" % row)
    p.chmod(0o755)
    return str(tmp_path)


@pytest.mark.parametrize("row,reasons", [
    ("0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active", []),
    ("0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active", ["sw_power_cap"]),
    ("0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Not Active", ["hw_slowdown"]),
])
def test_clock_sampler_window(tmp_path, monkeypatch, row, reasons):
    import bench
    monkeypatch.setenv("PATH", fake_smi(tmp_path, row) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0, period_ms=20).start()
    time.sleep(0.2)
    with s.window():
        time.sleep(0.15)
    s.stop()
    out = s.summary()
    f = [x.strip() for x in row.split(",")]
    assert out["sm_mhz"] == float(f[1]) and out["sm_max_mhz"] == float(f[2])
    assert out["reasons"] == reasons
    assert out["samples"] >= 2 and out["sampled"] == "timed region"


def test_clock_sampler_short_window_and_missing_tool(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", fake_smi(tmp_path, "0, 2070, 2070, 1.0, 0x0, Not Active, Not Active, "
                                                  "Not Active, Not Active") + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0, period_ms=20).start()
    time.sleep(0.2)
    with s.window():
        pass
    time.sleep(0.1)
    s.stop()
    assert s.summary()["sm_mhz"] == 2070.0
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    s = bench.ClockSampler(0).start()
    with s.window():
        pass
    s.stop()
    assert s.summary()["reasons"] == ["unsampled"]


def test_rollout_traffic_tracks_sources(tmp_path, monkeypatch):
    import bench
    v = bench.rollout_traffic()
    assert v is None or v == bench.ROLLOUT_TRAFFIC["bytes"]
    monkeypatch.setitem(bench.ROLLOUT_TRAFFIC, "sources_sha256", "0" * 16)
    assert bench.rollout_traffic() is None
