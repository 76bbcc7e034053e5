"""bench.py's clock sampler against a stand-in for nvidia-smi (no GPU needed).

The sampler must keep only the rows written after the timed region starts
(`Clocks.start`), take the median SM clock of those rows, and report the
throttle reasons that any of them shows active.
"""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# one row before the timed region (a low clock with hw_slowdown active), then
# rows under load; the pause after the first row lets start() see exactly one
# row, and its slowdown must not reach the report
FAKE = """#!/bin/sh
echo "0, 345, 2070, 100.0, Active, Active, Not Active, Not Active, Not Active"
sleep 0.2
i=0
while [ $i -lt 200 ]; do
  echo "0, 2070, 2070, 900.0, Active, Not Active, Not Active, Not Active, $CAP"
  sleep 0.02
  i=$((i + 1))
done
"""


def make_fake(tmp_path, cap):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(FAKE)
    f.chmod(f.stat().st_mode | stat.S_IEXEC)
    return str(d), cap


def run_sampler(monkeypatch, tmp_path, cap):
    d, cap = make_fake(tmp_path, cap)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.setenv("CAP", cap)
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.start()
    c.mark()
    time.sleep(0.7)
    return c.stop()


def test_rows_before_the_timed_region_are_dropped(monkeypatch, tmp_path):
    r = run_sampler(monkeypatch, tmp_path, "Not Active")
    assert r["samples"] >= 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == []


def test_active_throttle_reason_reported(monkeypatch, tmp_path):
    r = run_sampler(monkeypatch, tmp_path, "Active")
    assert r["reasons"] == ["sw_power_cap"]
    assert r["sm_mhz"] == 2070.0


def test_region_without_a_sample_falls_back_to_the_warm_up(monkeypatch, tmp_path):
    d, _ = make_fake(tmp_path, "Not Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.setenv("CAP", "Not Active")
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.start()            # the first row (hw_slowdown) is before the warm-up
    time.sleep(0.5)      # warm-up rows under load
    c.p.terminate()      # no row inside the timed region
    c.p.wait()
    c.mark()
    r = c.stop()
    assert r["samples"] == 0 and "warm-up" in r["note"]
    assert r["sm_mhz"] == 2070.0 and r["reasons"] == []


def test_missing_sampler(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.start()
    c.mark()
    r = c.stop()
    assert r["sm_mhz"] is None
