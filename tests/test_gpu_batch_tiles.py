"""Tiles of the lockstep batch's products (tomo_batch_set_tiles / tomo_batch_autotune_tiles):
4-row tiles and other wave targets solve every grid to the same tolerance as 8-row tiles
(only the dot partial order differs); the autotuner keeps the fastest candidate it timed;
the persistent iteration falls back to the launched one with 4-row tiles."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _fields(ps, seed):
    return [torch.tensor(P.random_field(p.dims, seed + i, 0.05, 1.0), dtype=torch.float32,
                         device=DEV) for i, p in enumerate(ps)]


def guarded_rel(x, ref):
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(x - ref) / den))


def _run(b, zs):
    dcs = [torch.empty_like(z) for z in zs]
    cs, infos = b.gradient(zs, dcs)
    torch.cuda.synchronize()
    return cs, [i.iters for i in infos], [d.cpu().numpy() for d in dcs]


def test_tile_settings_agree_and_are_validated():
    ps = P.uneven_cantilever_batch(21, 8)
    zs = _fields(ps, 700)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=4) as b:
            for g in grids:
                b.append(g)
            assert b.tiles() == (8, 4)
            ref = _run(b, zs)
            for bad in ((6, 4), (8, 0), (4, 17)):
                with pytest.raises(tomo.TomoError):
                    b.set_tiles(*bad)
            assert b.tiles() == (8, 4)
            for rows, waves in ((4, 4), (4, 1), (8, 8)):
                b.set_tiles(rows, waves)
                res = _run(b, zs)
                again = _run(b, zs)
                assert res[0] == again[0]                  # reproducible per setting
                for k in range(len(ps)):
                    assert abs(res[0][k] / ref[0][k] - 1.0) <= 1e-5
                    assert guarded_rel(res[2][k], ref[2][k]) <= 1e-4
                    assert abs(res[1][k] - ref[1][k]) <= 1
            b.set_tiles(4, 4)
            b.set_persistent(True)
            _run(b, zs)
            assert b.persistent_info[0] == 0               # launched iteration with 4 rows
            assert b.lockstep_runs == 8
    finally:
        for g in grids:
            g.close()


def test_tile_autotuner_keeps_the_fastest_candidate():
    ps = P.uneven_cantilever_batch(22, 6)
    zs = _fields(ps, 800)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=4) as b:
            for g in grids:
                b.append(g)
            dcs = [torch.empty_like(z) for z in zs]
            best, rows = b.autotune_tiles(zs, dcs, reps=2)
            assert [(r["rows"], r["waves"]) for r in rows] == [(8, 2), (8, 4), (8, 8),
                                                                (4, 2), (4, 4), (4, 8)]
            ok = [r for r in rows if r["status"] == 0]
            assert ok and all(r["ms"] > 0 for r in ok)
            fastest = min(ok, key=lambda r: r["ms"])
            assert best == (fastest["rows"], fastest["waves"]) and b.tiles() == best
            res = _run(b, zs)
        for g, z, c in zip(grids, zs, res[0]):
            dc = torch.empty_like(z)
            c0, _ = g.gradient(z, dc)
            assert abs(c / c0 - 1.0) <= 1e-5
    finally:
        for g in grids:
            g.close()
