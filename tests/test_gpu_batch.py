"""Batches of uneven grids (tomo_batch_*): each grid's result in the batch is the result it
gives alone, and agrees with the oracle; the 64-cantilever batch of uneven sizes runs
through one batch call."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _fields(ps, seed):
    return [torch.tensor(P.random_field(p.dims, seed + i, 0.05, 1.0), dtype=torch.float32,
                         device=DEV) for i, p in enumerate(ps)]


def test_batch_results_equal_results_alone():
    ps = P.uneven_cantilever_batch(3, 10)
    zs = _fields(ps, 100)
    alone = []
    for p, z in zip(ps, zs):
        with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
            dc = torch.empty_like(z)
            dv = torch.empty_like(z)
            c, info = g.gradient(z, dc, dv)
            torch.cuda.synchronize()
            alone.append((c, info.iters, dc.cpu().numpy(), dv.cpu().numpy()))
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=4) as b:
            for g in grids:
                b.append(g)
            assert len(b) == len(ps)
            dcs = [torch.empty_like(z) for z in zs]
            dvs = [torch.empty_like(z) for z in zs]
            for _ in range(2):   # twice: the second call reuses each grid's captured loop
                cs, infos = b.gradient(zs, dcs, dvs)
                torch.cuda.synchronize()
                for i, (c, it, dc, dv) in enumerate(alone):
                    assert cs[i] == c and infos[i].iters == it and infos[i].status == 0
                    assert np.array_equal(dcs[i].cpu().numpy(), dc)
                    assert np.array_equal(dvs[i].cpu().numpy(), dv)
    finally:
        for g in grids:
            g.close()


def test_batch_matches_oracle_on_the_smallest_grids():
    ps = sorted(P.uneven_cantilever_batch(5, 12), key=lambda p: p.n_el)[:3]
    zs = _fields(ps, 7)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=3) as b:
            for g in grids:
                b.append(g)
            dcs = [torch.empty_like(z) for z in zs]
            cs, infos = b.gradient(zs, dcs)
            torch.cuda.synchronize()
        for p, z, c, dc in zip(ps, zs, cs, dcs):
            ref = topopt.Model(p).gradient(z.cpu().numpy().astype(np.float64), "direct")
            assert abs(c / ref["c"] - 1.0) <= 1e-5
            d = dc.cpu().numpy().astype(np.float64)
            scale = np.abs(ref["dcdz"]).max()
            assert np.abs(d - ref["dcdz"]).max() <= 1e-4 * scale
    finally:
        for g in grids:
            g.close()


def test_batch_of_64_uneven_cantilevers_converges():
    ps = P.uneven_cantilever_batch(0, 64)
    sizes = [p.n_el for p in ps]
    assert min(sizes) >= 16 ** 3 and max(sizes) <= 64 * 32 * 32
    zs = [torch.full((p.n_el,), p.volfrac, dtype=torch.float32, device=DEV) for p in ps]
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=16) as b:
            for g in grids:
                b.append(g)
            dcs = [torch.empty_like(z) for z in zs]
            cs, infos = b.gradient(zs, dcs)
            torch.cuda.synchronize()
        assert all(i.status == 0 and i.rel_res <= 1e-6 for i in infos)
        assert all(np.isfinite(c) and c > 0 for c in cs)
        # spot-check one grid against its solve alone
        k = int(np.argmin(sizes))
        with tomo.Grid.from_problem(ps[k], precision=tomo.FP32) as g:
            dc = torch.empty_like(zs[k])
            c, _ = g.gradient(zs[k], dc)
        assert c == cs[k]
    finally:
        for g in grids:
            g.close()


def test_batch_rejects_fp64_grids():
    p = P.cantilever(8, 4, 4)
    with tomo.Grid.from_problem(p, precision=tomo.FP64) as g, tomo.Batch(workers=2) as b:
        b.append(g)
        z = torch.full((p.n_el,), 0.5, dtype=torch.float64, device=DEV)
        with pytest.raises((tomo.TomoError, TypeError)):
            b.gradient([z], [torch.empty_like(z)])


def test_batch_reports_the_failing_grid_and_finishes_the_others():
    ps = P.uneven_cantilever_batch(9, 4)
    zs = _fields(ps, 50)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32, maxit=(1 if i == 2 else 2000))
             for i, p in enumerate(ps)]
    try:
        with tomo.Batch(workers=2) as b:
            for g in grids:
                b.append(g)
            dcs = [torch.empty_like(z) for z in zs]
            with pytest.raises(tomo.TomoError) as ei:
                b.gradient(zs, dcs)
            assert "grid 2" in str(ei.value)
        torch.cuda.synchronize()
        # the grids that converged hold their results
        for i in (0, 1, 3):
            with tomo.Grid.from_problem(ps[i], precision=tomo.FP32) as g:
                dc = torch.empty_like(zs[i])
                g.gradient(zs[i], dc)
            assert torch.equal(dc, dcs[i])
    finally:
        for g in grids:
            g.close()
