"""Clock sampling in bench.py, driven by a fake nvidia-smi on the CPU: the sampler waits for
its first row before the timed region, keeps sampling until exit, falls back to a longer
interval when the short one is refused, and reports throttle reasons it sees."""
import os
import stat
import sys
import time

import bench

FAKE = r'''#!{python}
import os, sys, time
ms = int(sys.argv[sys.argv.index("-lms") + 1])
if os.environ.get("FAKE_SMI_REJECT") == str(ms):
    sys.stderr.write("invalid interval\n")
    sys.exit(2)
cap = "Active" if os.environ.get("FAKE_SMI_POWERCAP") else "Not Active"
time.sleep(float(os.environ.get("FAKE_SMI_STARTUP", "0")))
while True:
    print(f"0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {{cap}}", flush=True)
    time.sleep(ms / 1000.0)
'''


def fake_smi(tmp_path):
    path = tmp_path / "fake-nvidia-smi"
    path.write_text(FAKE.format(python=sys.executable))
    path.chmod(path.stat().st_mode | stat.S_IEXEC)
    return str(path)


def test_samples_through_a_short_timed_region(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_SMI_STARTUP", "0.3")
    with bench.ClockSampler(0, exe=fake_smi(tmp_path)) as clk:
        assert clk.rows, "entering returns only after the first row"
        time.sleep(0.3)
    s = clk.summary()
    assert s["interval_ms"] == 50
    assert s["samples"] >= 4
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == []
    assert clk.proc.poll() is not None


def test_falls_back_when_the_short_interval_is_refused(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_SMI_REJECT", "50")
    with bench.ClockSampler(0, exe=fake_smi(tmp_path)) as clk:
        time.sleep(0.05)
    s = clk.summary()
    assert s["interval_ms"] == 200
    assert s["samples"] >= 1


def test_power_cap_is_reported(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_SMI_POWERCAP", "1")
    with bench.ClockSampler(0, exe=fake_smi(tmp_path)) as clk:
        pass
    assert clk.summary()["reasons"] == ["sw_power_cap"]


def test_missing_sampler_reads_unsampled(tmp_path):
    with bench.ClockSampler(0, exe=os.path.join(str(tmp_path), "absent")) as clk:
        pass
    assert clk.summary()["reasons"] == ["unsampled"]
