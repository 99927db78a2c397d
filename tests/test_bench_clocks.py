"""bench.py's clock sampler on the host, against a stand-in nvidia-smi put first on PATH: it
keeps only the samples whose timestamps fall inside the marked timed windows (a throttle
reason seen before the window is not reported), falls back to every sample when the
timestamps do not parse, and reports nothing, without failing, when nvidia-smi is absent.
No GPU is needed."""
import os
import stat
import sys
import time

import bench

FAKE = r'''#!{py}
import datetime, sys, time
t0 = time.time()
while True:
    now = time.time()
    stamp = "n/a" if {garbled} else datetime.datetime.fromtimestamp(now).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    cap = "Active" if now - t0 < 0.3 else "Not Active"
    print(f"{{stamp}}, 0, 1980, 2070, 850.0, 0x0000000000000004, Not Active, Not Active, Not Active, {{cap}}",
          flush=True)
    time.sleep(0.02)
'''


def _fake(tmp_path, monkeypatch, garbled):
    p = tmp_path / "nvidia-smi"
    p.write_text(FAKE.format(py=sys.executable, garbled=garbled))
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))


def _run():
    with bench.ClockSampler(0) as clk:
        time.sleep(0.8)                  # the stand-in reports a power cap for its first 0.3 s
        clk.mark_start()
        time.sleep(0.4)
        clk.mark_end()
        time.sleep(0.1)
    return clk.summary()


def test_keeps_only_samples_inside_the_timed_window(tmp_path, monkeypatch):
    _fake(tmp_path, monkeypatch, garbled=False)
    s = _run()
    assert s["window"] == "timed region"
    assert 5 <= s["samples"] <= 30
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []


def test_falls_back_to_every_sample_without_timestamps(tmp_path, monkeypatch):
    _fake(tmp_path, monkeypatch, garbled=True)
    s = _run()
    assert s["window"].startswith("whole sampling")
    assert s["samples"] >= 20 and s["reasons"] == ["sw_power_cap"]


def test_absent_nvidia_smi_reports_nothing(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    with bench.ClockSampler(0) as clk:
        clk.mark_start()
        clk.mark_end()
    s = clk.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []
