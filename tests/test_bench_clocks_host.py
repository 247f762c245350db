"""The benchmark's clock sampler (the nvidia-smi process that records SM clocks and
throttle reasons around the timed legs), run against a stand-in nvidia-smi on the host:
start() returns only once the first sample has arrived, so the sampler's start-up lands
before any timed leg; the summary takes the median SM clock and every active reason, and
reports "unavailable" when no nvidia-smi runs."""
import os
import stat
import time

import bench

# a stand-in that starts slowly and then prints one sample per 50 ms in the query's
# column order: index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
FAKE = """#!/bin/sh
sleep 0.3
for c in 1965 2070 2070 1950 2070 2070; do
  echo "0, $c, 2070, 980.25, 0x4, Not Active, Not Active, Not Active, Active"
  sleep 0.05
done
exec sleep 30
"""


def _fake_smi(tmp_path, monkeypatch, body):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(body)
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ.get('PATH', '')}")


def test_start_waits_for_the_first_sample_and_summary_reads_reasons(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch, FAKE)
    c = bench.ClockSampler("GPU-test")
    t0 = time.time()
    c.start()
    assert c.rows, "start() returned before the first sample"
    assert time.time() - t0 >= 0.25
    time.sleep(0.4)
    c.stop()
    assert c.proc.poll() is not None  # the stand-in was terminated
    s = c.summary(0.0, time.time())
    assert s["samples"] == 6
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_a_sampler_that_prints_nothing_does_not_hold_the_benchmark(tmp_path, monkeypatch):
    _fake_smi(tmp_path, monkeypatch, "#!/bin/sh\nexit 3\n")
    c = bench.ClockSampler("GPU-test")
    t0 = time.time()
    c.start()
    assert time.time() - t0 < 5.0  # the process ended: no wait for the full deadline
    c.stop()
    assert c.summary(0.0, time.time()) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"],
                                           "samples": 0}


def test_no_nvidia_smi_at_all(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory
    c = bench.ClockSampler("GPU-test")
    c.start()
    c.stop()
    assert c.proc is None and c.summary(0.0, time.time())["reasons"] == ["unavailable"]
