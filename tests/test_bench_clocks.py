"""The benchmark's clock record on CPU, against a stand-in nvidia-smi that
prints one query row every 50 ms: the samples counted are those written
while the caller's region runs, and a region shorter than the interval
reports the nearest sample, flagged as outside the region."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!{py}
import sys, time
time.sleep(0.2)
i = 0
while True:
    reason = "Active" if i >= {slow_from} else "Not Active"
    print("0, %d, 2070, 900.0, 0x0, Not Active, %s, Not Active, Not Active" % (1900 if i >= {slow_from} else 2070, reason),
          flush=True)
    i += 1
    time.sleep(0.05)
"""


def _sampler(tmp_path, monkeypatch, slow_from=10 ** 9):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(FAKE.format(py=sys.executable, slow_from=slow_from))
    f.chmod(f.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(d) + os.pathsep + os.environ.get("PATH", ""))
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    return bench.ClockSampler(0)


def test_samples_fall_inside_the_region(tmp_path, monkeypatch):
    c = _sampler(tmp_path, monkeypatch)
    c.start()
    assert c.skip >= 1              # the sampler was live before the region began
    time.sleep(0.6)
    ck = c.stop()
    assert ck["in_region"] and ck["samples"] >= 5
    assert ck["sm_mhz"] == 2070.0 and ck["sm_max_mhz"] == 2070.0 and ck["reasons"] == []


def test_short_region_reports_the_nearest_sample(tmp_path, monkeypatch):
    c = _sampler(tmp_path, monkeypatch)
    c.start()
    ck = c.stop()
    assert ck["samples"] == 1 and not ck["in_region"]


def test_slowdown_inside_the_region_is_reported(tmp_path, monkeypatch):
    c = _sampler(tmp_path, monkeypatch, slow_from=3)
    c.start()
    time.sleep(0.6)
    ck = c.stop()
    assert ck["in_region"]
    assert "hw_thermal_slowdown" in ck["reasons"]
    assert ck["sm_mhz"] == 1900.0


def test_missing_nvidia_smi_gives_no_record(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() is None
