"""bench.py's clock sampler on CPU, against a stand-in nvidia-smi that prints one CSV line every
50 ms: only the lines read from one period before start() to one period after stop() count, the
throttle reasons are parsed from their columns, and a missing nvidia-smi is reported, not raised."""
import importlib.util
import os
import stat
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_smi(tmp_path, line):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(f"#!/bin/sh\nwhile true; do echo '{line}'; sleep 0.05; done\n")
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_samples_in_the_window_and_reasons(tmp_path, monkeypatch):
    line = "0, 1980, 2070, 1200.5, 0x4, Not Active, Not Active, Not Active, Active"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, line) + os.pathsep + os.environ["PATH"])
    b = _bench()
    monkeypatch.setattr(b.ClockSampler, "PERIOD_S", 0.05)
    c = b.ClockSampler(0)
    time.sleep(0.5)  # lines read long before start() are not counted
    c.start()
    time.sleep(0.3)
    out = c.stop()
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    # 0.3 s region + one 50 ms period on each side: about 8 lines, never the ~10 read before
    assert 3 <= out["samples"] <= 10, out
    assert 0.29 <= out["timed_region_s"] <= 0.5


def test_missing_nvidia_smi_is_reported(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory: no nvidia-smi
    b = _bench()
    c = b.ClockSampler(0)
    c.start()
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
