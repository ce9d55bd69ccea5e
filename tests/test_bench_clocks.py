"""The benchmark's clock sampler against a stand-in for nvidia-smi on PATH
(CPU only): samples are taken while the timed region runs, the median SM
clock, the maximum clock and the active throttle reasons are read from them,
and without nvidia-smi the sampler reports nothing instead of failing."""

import os
import stat
import time

FAKE = """#!/bin/sh
# stand-in for nvidia-smi --query-gpu=... --format=csv,noheader,nounits -lms N
while true; do
  echo "0, 1965, 2070, 700.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
  sleep 0.02
done
"""


def test_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE)
    exe.chmod(exe.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    import bench
    s = bench.ClockSampler(0, interval_ms=20)
    s.start()
    time.sleep(0.2)
    r = s.stop()
    assert r is not None and r["samples"] >= 3
    assert r["sm_mhz"] == 1965.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["interval_ms"] == 20


def test_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    import bench
    s = bench.ClockSampler(0)
    t0 = time.time()
    s.start()
    assert s.stop() is None
    assert time.time() - t0 < 1.0
