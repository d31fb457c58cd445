"""Batches of uneven grids (tomo_batch_*): one grid per stream, each grid's result is
bitwise the result it gives alone; in lockstep (one CG loop for all grids, one launch per
phase) it agrees with the result alone to the solver's tolerance and is reproducible; both
agree with the oracle; the 64-cantilever batch of uneven sizes runs through one call."""
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


def guarded_rel(x, ref):
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(x - ref) / den))


def close(c, dc, c0, dc0):
    """Two solves of the same system to rtol 1e-6 (different rounding of the CG dots): the
    stated tolerances, compliance 1e-5 relative and sensitivities 1e-4 guarded."""
    return abs(c / c0 - 1.0) <= 1e-5 and guarded_rel(np.asarray(dc, np.float64),
                                                     np.asarray(dc0, np.float64)) <= 1e-4


@pytest.mark.parametrize("lockstep", [False, True])
def test_batch_results_equal_results_alone(lockstep):
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
        with tomo.Batch(workers=4, lockstep=lockstep) as b:
            for g in grids:
                b.append(g)
            assert len(b) == len(ps)
            dcs = [torch.empty_like(z) for z in zs]
            dvs = [torch.empty_like(z) for z in zs]
            first = None
            for _ in range(2):   # twice: the second call reuses the captured loop(s)
                cs, infos = b.gradient(zs, dcs, dvs)
                torch.cuda.synchronize()
                got = (cs, [d.cpu().numpy() for d in dcs])
                for i, (c, it, dc, dv) in enumerate(alone):
                    assert infos[i].status == 0
                    assert np.array_equal(dvs[i].cpu().numpy(), dv)
                    if lockstep:
                        assert close(cs[i], got[1][i], c, dc) and abs(infos[i].iters - it) <= 1
                    else:
                        assert cs[i] == c and infos[i].iters == it
                        assert np.array_equal(got[1][i], dc)
                if first is None:
                    first = got
                else:   # reproducible
                    assert got[0] == first[0]
                    assert all(np.array_equal(a, b2) for a, b2 in zip(got[1], first[1]))
            assert b.lockstep_runs == (2 if lockstep else 0)
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
        assert close(cs[k], dcs[k].cpu().numpy(), c, dc.cpu().numpy())
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
                c, _ = g.gradient(zs[i], dc)
            assert guarded_rel(dcs[i].cpu().numpy().astype(np.float64),
                               dc.cpu().numpy().astype(np.float64)) <= 1e-4
    finally:
        for g in grids:
            g.close()


def _run_batch(grids, zs, lockstep, workers=4, repeat=1):
    with tomo.Batch(workers=workers, lockstep=lockstep) as b:
        for g in grids:
            b.append(g)
        dcs = [torch.empty_like(z) for z in zs]
        dvs = [torch.empty_like(z) for z in zs]
        for _ in range(repeat):
            cs, infos = b.gradient(zs, dcs, dvs)
        torch.cuda.synchronize()
        runs = b.lockstep_runs
    return cs, infos, [d.cpu().numpy() for d in dcs], [d.cpu().numpy() for d in dvs], runs


def test_lockstep_loop_agrees_with_one_grid_per_stream():
    """The lockstep loop (one launch per phase for all grids, grids of 3 to 5 multigrid
    levels) agrees with the grids run one per stream, and repeats itself exactly."""
    ps = P.uneven_cantilever_batch(11, 12)
    zs = _fields(ps, 300)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        assert len({g.counts()[2] for g in grids}) > 1     # uneven level counts
        a = _run_batch(grids, zs, lockstep=False)
        b = _run_batch(grids, zs, lockstep=True, repeat=2)
        b2 = _run_batch(grids, zs, lockstep=True)
        assert a[4] == 0 and b[4] == 2 and b2[4] == 1
        for k in range(len(ps)):
            assert close(b[0][k], b[2][k], a[0][k], a[2][k])
            assert abs(a[1][k].iters - b[1][k].iters) <= 1
            assert np.array_equal(a[3][k], b[3][k])          # dV/dz: no solve involved
        assert b[0] == b2[0] and all(np.array_equal(x, y) for x, y in zip(b[2], b2[2]))
    finally:
        for g in grids:
            g.close()


def test_lockstep_with_a_zero_load_grid_and_residual_replacement():
    """A grid with no load (solution 0, no CG iteration) sits in the batch beside grids
    whose solves replace the residual every 4 iterations (the batched FP64 residual)."""
    ps = P.uneven_cantilever_batch(12, 5)
    ps[1].f[:] = 0.0
    zs = _fields(ps, 400)
    alone = []
    for p, z in zip(ps, zs):
        with tomo.Grid.from_problem(p, precision=tomo.FP32, rr_every=4) as g:
            dc = torch.empty_like(z)
            c, info = g.gradient(z, dc)
            torch.cuda.synchronize()
            alone.append((c, info.iters, dc.cpu().numpy()))
    assert alone[1][0] == 0.0 and alone[1][1] == 0
    assert max(a[1] for a in alone) > 8
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32, rr_every=4) for p in ps]
    try:
        cs, infos, dcs, _, runs = _run_batch(grids, zs, lockstep=True)
        assert runs == 1
        assert cs[1] == 0.0 and infos[1].iters == 0 and not np.any(dcs[1])
        for k, ((c, it, dc), c2, i2, dc2) in enumerate(zip(alone, cs, infos, dcs)):
            if k != 1:
                assert close(c2, dc2, c, dc) and abs(it - i2.iters) <= 1
    finally:
        for g in grids:
            g.close()


def test_lockstep_warm_starts_follow_the_grids_alone():
    ps = P.uneven_cantilever_batch(13, 4)
    z1, z2 = _fields(ps, 500), _fields(ps, 600)
    alone = []
    for p, a, b in zip(ps, z1, z2):
        with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
            g.set_warm_start(True)
            dc = torch.empty_like(a)
            g.gradient(a, dc)
            c, info = g.gradient(b, dc)
            torch.cuda.synchronize()
            alone.append((c, info.iters, dc.cpu().numpy()))
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        for g in grids:
            g.set_warm_start(True)
        with tomo.Batch(workers=2) as bt:
            for g in grids:
                bt.append(g)
            dcs = [torch.empty_like(z) for z in z1]
            bt.gradient(z1, dcs)
            cs, infos = bt.gradient(z2, dcs)
            torch.cuda.synchronize()
            assert bt.lockstep_runs == 2
        for (c, it, dc), c2, i2, d2 in zip(alone, cs, infos, dcs):
            assert close(c2, d2.cpu().numpy(), c, dc) and abs(it - i2.iters) <= 1
    finally:
        for g in grids:
            g.close()


def test_batch_of_different_poisson_ratios_runs_per_stream():
    ps = P.uneven_cantilever_batch(14, 3)
    ps[2].nu = 0.25
    zs = _fields(ps, 700)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        cs, infos, dcs, _, runs = _run_batch(grids, zs, lockstep=True)
        assert runs == 0                     # not lockstep-compatible: one grid per stream
        with tomo.Grid.from_problem(ps[2], precision=tomo.FP32) as g:
            dc = torch.empty_like(zs[2])
            c, _ = g.gradient(zs[2], dc)
        assert c == cs[2] and np.array_equal(dc.cpu().numpy(), dcs[2])
    finally:
        for g in grids:
            g.close()


def test_lockstep_with_host_arrays():
    """Host (numpy) arrays go through the grids' staging buffers in lockstep too."""
    ps = P.uneven_cantilever_batch(15, 3)
    zh = [P.random_field(p.dims, 800 + i, 0.05, 1.0).astype(np.float32)
          for i, p in enumerate(ps)]
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=2) as b:
            for g in grids:
                b.append(g)
            dch = [np.zeros(p.n_el, np.float32) for p in ps]
            dvh = [np.zeros(p.n_el, np.float32) for p in ps]
            cs, infos = b.gradient(zh, dch, dvh)
            assert b.lockstep_runs == 1
            zd = [torch.tensor(z, device=DEV) for z in zh]
            dcd = [torch.empty_like(z) for z in zd]
            cs2, _ = b.gradient(zd, dcd)
            torch.cuda.synchronize()
        for c, c2, a, d in zip(cs, cs2, dch, dcd):
            assert c == c2 and np.array_equal(a, d.cpu().numpy())
        assert all(np.all(v > 0) for v in dvh)
    finally:
        for g in grids:
            g.close()


def test_lockstep_with_very_different_hierarchies():
    """Grids of 2 to 6 multigrid levels and both problem types in one lockstep loop: each
    grid's coarsest solve comes after the batch's down-sweep."""
    ps = [P.cantilever(4, 2, 2), P.mbb_block(96, 48, 40, volfrac=0.12, rmin=2.5),
          P.cantilever(9, 5, 3), P.mbb_block(33, 17, 9, rmin=1.5), P.cantilever(64, 32, 32)]
    zs = _fields(ps, 900)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        levels = [g.counts()[2] for g in grids]
        assert min(levels) == 2 and max(levels) >= 6
        alone = []
        for g, z in zip(grids, zs):
            dc = torch.empty_like(z)
            c, info = g.gradient(z, dc)
            torch.cuda.synchronize()
            alone.append((c, info.iters, dc.cpu().numpy()))
        cs, infos, dcs, _, runs = _run_batch(grids, zs, lockstep=True, workers=3)
        assert runs == 1
        for (c, it, dc), c2, i2, d2 in zip(alone, cs, infos, dcs):
            assert i2.status == 0 and close(c2, d2, c, dc) and abs(it - i2.iters) <= 1
    finally:
        for g in grids:
            g.close()
