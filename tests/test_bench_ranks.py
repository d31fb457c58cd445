"""Replica timing across ranks (the N > 1 path of bench.py) on CPU with gloo, world size 2.

The path has no exchange step: every rank runs its own replica, the process group only
brackets the timed region and takes the slowest rank's time.  These tests run that host
logic with two gloo processes on 127.0.0.1 (no GPU)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
dist = bench.init_ranks("gloo")
world, rank, _ = bench.dist_env()
local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
dist.barrier()
slowest = bench.max_over_ranks(dist, local_ms)
value = bench.whole_job_rate(world, 10, slowest)
with open(os.path.join({out!r}, f"rank{{rank}}.json"), "w") as fh:
    json.dump({{"rank": rank, "world": world, "slowest": slowest, "value": value}}, fh)
dist.destroy_process_group()
"""


def _launch(tmp_path, world):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        code = _CHILD.format(root=ROOT, out=str(tmp_path))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env))
    for p in procs:
        assert p.wait(timeout=120) == 0
    return [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    res = _launch(tmp_path, 2)
    for r in res:
        assert r["world"] == 2
        assert r["slowest"] == pytest.approx(200.0)
        # 2 ranks x 10 steps in 0.2 s (the slowest rank) = 100 steps/s for the whole job
        assert r["value"] == pytest.approx(100.0)


def test_single_process_needs_no_group(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.init_ranks("gloo") is None
    assert bench.max_over_ranks(None, 12.5) == 12.5
    assert bench.whole_job_rate(1, 20, 1000.0) == pytest.approx(20.0)


def test_reference_arm_prints_on_rank0_only(monkeypatch, capsys):
    class Args:
        gpus, steps, warmup, seed = 2, 1, 0, 0
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
