"""Host logic of bench.py that needs no GPU: the clock sampler keeps the nvidia-smi samples
whose timestamps fall inside the timed region (a stand-in nvidia-smi prints them here), and
reports its absence instead of failing."""

import importlib.util
import os
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_sampler_keeps_only_samples_inside_the_timed_region(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/bash\nwhile true; do\n"
                    "  echo \"$(date +'%Y/%m/%d %H:%M:%S.%3N'), 0, 1980, 2070, 900.0, 0x4, "
                    "Not Active, Not Active, Not Active, Active\"\n  sleep 0.02\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = _bench().ClockSampler(0)
    c.start()
    time.sleep(0.3)  # samples before the region
    c.begin()
    time.sleep(0.3)
    c.end()
    time.sleep(0.3)  # and after it
    r = c.stop()
    total = len(c.lines)
    assert 3 <= r["samples"] < total, (r, total)
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert 250 <= r["window_ms"] <= 600


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = _bench().ClockSampler(0)
    c.start()
    c.begin()
    c.end()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
