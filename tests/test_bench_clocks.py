"""Clock sampling in bench.py, driven by a fake nvidia-smi on the CPU: the sampler is up
before the timed region, summarises only rows from the region's start (marked), waits for
one row when the region is shorter than an interval, falls back to a longer interval when
the short one is refused, and reports the throttle reasons it sees."""
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
k = 0
while True:  # the k-th row reads an SM clock of 1000 + k MHz
    print(f"0, {{1000 + k}}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {{cap}}",
          flush=True)
    k += 1
    time.sleep(ms / 1000.0)
'''


def fake_smi(tmp_path):
    path = tmp_path / "fake-nvidia-smi"
    path.write_text(FAKE.format(python=sys.executable))
    path.chmod(path.stat().st_mode | stat.S_IEXEC)
    return str(path)


def test_rows_before_the_timed_region_are_dropped(tmp_path, monkeypatch):
    monkeypatch.setenv("FAKE_SMI_STARTUP", "0.3")
    with bench.ClockSampler(0, exe=fake_smi(tmp_path)) as clk:
        assert clk._rows, "entering returns only after the first row"
        time.sleep(0.2)  # warm-up steps
        clk.mark()
        first = clk.first
        assert first >= 1
        time.sleep(0.3)  # timed steps
    s = clk.summary()
    assert s["interval_ms"] == 50
    assert s["samples"] >= 2
    assert min(float(r[1]) for r in clk.rows) == 1000 + first
    assert s["sm_max_mhz"] == 2070.0 and s["reasons"] == []
    assert clk.proc.poll() is not None


def test_a_region_shorter_than_an_interval_waits_for_one_row(tmp_path):
    with bench.ClockSampler(0, exe=fake_smi(tmp_path)) as clk:
        clk.mark()
    assert clk.summary()["samples"] >= 1
    assert float(clk.rows[0][1]) >= 1000 + clk.first


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
