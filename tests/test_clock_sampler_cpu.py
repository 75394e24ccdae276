"""The bench's clock record (median SM clock under load, the maximum, and the throttle reasons seen),
checked without a GPU against a stand-in nvidia-smi that prints fixed samples."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

ROWS = [
    "0, 1980, 2070, 1200.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2070, 2070, 1300.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2070, 2070, 1310.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, [N/A], 2070, 1310.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
]


def _fake_smi(tmp_path, rows):
    path = tmp_path / "nvidia-smi"
    path.write_text("#!/bin/sh\ncat <<'EOF'\n" + "\n".join(rows) + "\nEOF\n")
    path.chmod(path.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def _sample(monkeypatch, tmp_path, rows):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    time.sleep(0.5)
    return s.stop()


def test_median_clock_and_power_cap_reason(monkeypatch, tmp_path):
    rec = _sample(monkeypatch, tmp_path, ROWS)
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0      # median of the three numeric samples
    assert rec["reasons"] == ["sw_power_cap"]


def test_thermal_and_hardware_slowdowns_are_reported(monkeypatch, tmp_path):
    rows = ["0, 1500, 2070, 1400.0, 0x0000000000000048, Active, Not Active, Active, Not Active",
            "0, 1600, 2070, 1400.0, 0x0000000000000020, Not Active, Active, Not Active, Not Active"]
    rec = _sample(monkeypatch, tmp_path, rows)
    assert rec["sm_mhz"] == 1550.0
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_no_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))                          # no nvidia-smi anywhere on PATH
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ClockSampler(0).stop() is None
