"""The bounds-checked build (libtomo_checked.so, -DTOMO_CHECKED) records no index outside
its buffer on small and odd grids and every feature of the path, and gives the regular
build's results (tests/checked_workload.py run against each build in its own process)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(lib):
    env = dict(os.environ)
    env.pop("TOMO_LIB", None)
    if lib:
        env["TOMO_LIB"] = lib
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_workload.py")],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_finds_no_violation_and_agrees():
    from paper_2104_12282_gb300 import _build
    if not os.path.exists(_build.LIB_CHECKED):
        _build.build(checked=True)
    chk = _run("checked")
    reg = _run(None)
    assert chk["checked"] is True and reg["checked"] is False
    assert chk["word"] == 0, "site %d index %d" % (chk["word"] >> 48, chk["word"] & (2**48 - 1))
    assert chk["results"].keys() == reg["results"].keys()
    for k, v in reg["results"].items():
        w = chk["results"][k]
        for a, b in zip(v, w):
            assert abs(a - b) <= 1e-6 * max(abs(a), 1e-30) or a == b, (k, v, w)
