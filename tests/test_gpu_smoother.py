"""Smoother settings and the smoother autotuner (tomo_set_smoother, tomo_autotune_smoother):
every setting solves the same system to the same tolerance (checked against the oracle's
direct solve); the autotuner keeps the fastest converging candidate it timed; a lockstep
batch follows a smoother change of its grids."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _field(p, seed):
    z = P.random_field(p.dims, seed, 0.05, 1.0).astype(np.float32)
    return z, torch.tensor(z, device=DEV)


@pytest.mark.parametrize("degs", [(2, 2), (1, 4), (3, 6), (1, 1)])
def test_every_smoother_solves_to_tolerance(degs):
    p = P.cantilever(24, 12, 12)
    z, zt = _field(p, 31)
    ref = topopt.Model(p).gradient(z.astype(np.float64), "direct")
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        g.set_smoother(*degs)
        assert g.smoother()[:2] == degs
        dc = torch.empty_like(zt)
        c, info = g.gradient(zt, dc)
    assert info.status == 0 and info.rel_res <= 1e-6
    assert abs(c / ref["c"] - 1.0) <= 1e-5
    d = dc.cpu().numpy().astype(np.float64)
    assert np.abs(d - ref["dcdz"]).max() <= 1e-4 * np.abs(ref["dcdz"]).max()


def test_smoother_settings_change_iterations():
    p = P.mbb_block(48, 24, 19, volfrac=0.12, rmin=2.5)
    _, zt = _field(p, 32)
    its = {}
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        dc = torch.empty_like(zt)
        for degs in ((1, 1), (2, 2), (2, 6)):
            g.set_smoother(*degs)
            _, info = g.gradient(zt, dc)
            its[degs] = info.iters
    assert its[(1, 1)] > its[(2, 2)] >= its[(2, 6)]


def test_bad_smoother_values_are_rejected():
    p = P.cantilever(8, 4, 4)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        before = g.smoother()
        for args in ((0, 2, 20.0), (2, 17, 20.0), (2, 2, 1.0), (2, 2, float("nan"))):
            with pytest.raises(tomo.TomoError) as e:
                g.set_smoother(*args)
            assert e.value.status == 1
        assert g.smoother() == before


def test_autotune_keeps_the_fastest_converging_candidate():
    p = P.mbb_block(48, 24, 19, volfrac=0.12, rmin=2.5)
    z, zt = _field(p, 33)
    cands = [(2, 2), (1, 4), (2, 4), (1, 1)]
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        best, rows = g.autotune(zt, cands, reps=2)
        assert [(r["fine"], r["coarse"]) for r in rows] == cands
        ok = [r for r in rows if r["status"] == 0]
        assert ok and all(r["ms"] > 0 for r in ok)
        fastest = min(ok, key=lambda r: r["ms"])
        assert best == (fastest["fine"], fastest["coarse"], fastest["lam"], 0, 20.0)
        assert g.smoother()[:2] == best[:2] and g.smoother_bound()[0] == best[2]
        dc = torch.empty_like(zt)
        c, info = g.gradient(zt, dc)
        assert info.iters == fastest["iters"]
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g0:
        dc0 = torch.empty_like(zt)
        c0, _ = g0.gradient(zt, dc0)
    assert abs(c / c0 - 1.0) <= 1e-5
    # the built-in list
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        best, rows = g.autotune(zt)
        lam_b = g.smoother_bound()[1]
        assert len(rows) == 23
        assert best in [(r["fine"], r["coarse"], r["lam"], r["w"], r["ratio"]) for r in rows]
        assert sorted({round(r["lam"] / lam_b, 6) for r in rows}) == [0.68, 0.75, 1.0]
        assert [r["w"] for r in rows[:20]] == [0] * 18 + [2, 6]
        assert [r["ratio"] for r in rows[20:]] == [12.0, 30.0, 50.0]
        v = [r for r in rows[:18] if r["status"] == 0]
        vbest = min(v, key=lambda r: r["ms"])       # the W stage starts from the best V row
        assert all((r["fine"], r["coarse"], r["lam"]) == (vbest["fine"], vbest["coarse"],
                                                          vbest["lam"]) for r in rows[18:20])
        wbest = min([r for r in rows[:20] if r["status"] == 0], key=lambda r: r["ms"])
        assert all((r["fine"], r["coarse"], r["lam"], r["w"]) ==
                   (wbest["fine"], wbest["coarse"], wbest["lam"], wbest["w"])
                   for r in rows[20:])                # the ratio stage from the best so far
        assert g.smoother_bound()[0] == best[2] and g.cycle() == best[3]
        assert g.smoother()[2] == best[4]
        dc = torch.empty_like(zt)
        c2, _ = g.gradient(zt, dc)
    assert abs(c2 / c0 - 1.0) <= 1e-5


def test_autotune_over_several_designs_sums_their_times():
    p = P.mbb_block(48, 24, 19, volfrac=0.12, rmin=2.5)
    zs = [_field(p, 40 + k)[1] for k in range(3)]
    cands = [(2, 2), (1, 4)]
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        best, rows = g.autotune(zs, cands, reps=2)
        assert len(rows) == 2 and all(r["status"] == 0 and r["ms"] > 0 for r in rows)
        fastest = min(rows, key=lambda r: r["ms"])
        assert best[:2] == (fastest["fine"], fastest["coarse"])
        one = [g.autotune(z, cands, reps=2)[1] for z in zs]
        for k in range(2):    # the sum of three medians: larger than any one of them
            assert rows[k]["ms"] > max(o[k]["ms"] for o in one) * 1.5
            assert rows[k]["iters"] == max(o[k]["iters"] for o in one)
        with pytest.raises(tomo.TomoError):
            g.autotune([], cands)


def test_autotune_without_a_converging_candidate_keeps_the_smoother():
    p = P.cantilever(24, 12, 12)
    _, zt = _field(p, 34)
    with tomo.Grid.from_problem(p, precision=tomo.FP32, maxit=1) as g:
        g.set_smoother(2, 3)
        with pytest.raises(tomo.TomoError) as e:
            g.autotune(zt, [(1, 1), (2, 2)], reps=1)
        assert e.value.status == 3
        assert g.smoother()[:2] == (2, 3)


def test_lockstep_batch_follows_a_smoother_change():
    ps = P.uneven_cantilever_batch(21, 4)
    zs = [torch.tensor(P.random_field(p.dims, 40 + i, 0.05, 1.0), dtype=torch.float32,
                       device=DEV) for i, p in enumerate(ps)]
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=2) as b:
            for g in grids:
                b.append(g)
            dcs = [torch.empty_like(z) for z in zs]
            _, i0 = b.gradient(zs, dcs)
            grids[0].set_smoother(1, 4)          # grids now differ: one per stream
            b.gradient(zs, dcs)
            assert b.lockstep_runs == 1
            for g in grids[1:]:
                g.set_smoother(1, 4)             # the same again: lockstep, new loop
            cs, i1 = b.gradient(zs, dcs)
            assert b.lockstep_runs == 2
            torch.cuda.synchronize()
        for p, z, c, dc, info in zip(ps, zs, cs, dcs, i1):
            with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
                g.set_smoother(1, 4)
                d0 = torch.empty_like(z)
                c0, info0 = g.gradient(z, d0)
            assert abs(c / c0 - 1.0) <= 1e-5 and abs(info.iters - info0.iters) <= 1
    finally:
        for g in grids:
            g.close()


def test_smoother_bound_is_checked_and_a_failing_bound_falls_back():
    p = P.cantilever(24, 12, 12)
    z, zt = _field(p, 35)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g0:
        dc0 = torch.empty_like(zt)
        c0, info0 = g0.gradient(zt, dc0)
        lam_b = g0.smoother_bound()[1]
        assert g0.smoother_bound() == (lam_b, lam_b, 0) and 5.0 < lam_b < 5.5
        for bad in (0.2 * lam_b, 1.01 * lam_b, float("nan")):
            with pytest.raises(tomo.TomoError) as e:
                g0.set_smoother_bound(bad)
            assert e.value.status == 1
        g0.set_smoother_bound(0.0)                 # <= 0: the element bound
        assert g0.smoother_bound()[0] == lam_b
    # far below the spectrum of D^-1 K: the solve at that bound cannot converge within a
    # few iterations more than the element bound needs, so it is redone at the bound
    with tomo.Grid.from_problem(p, precision=tomo.FP32, maxit=info0.iters + 3) as g:
        g.set_smoother_bound(0.25 * lam_b)
        dc = torch.empty_like(zt)
        c, info = g.gradient(zt, dc)
        lam, _, falls = g.smoother_bound()
        assert info.status == 0
        assert (falls == 1 and lam == lam_b) or (falls == 0 and lam == 0.25 * lam_b)
        assert abs(c / c0 - 1.0) <= 1e-5
