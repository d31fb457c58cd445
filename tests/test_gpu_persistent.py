"""Persistent lockstep iteration (tomo_batch_set_persistent): each CG iteration of the
lockstep loop as one cooperative launch whose phases are the recorded batched launches.
Every grid runs the same blocks with the same dot-partial order as in the launched loop, so
the results are bitwise those of the launched lockstep loop; a barrier wait that runs out
stops the loop with TOMO_ETIMEOUT and leaves the context and the batch usable."""
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


def _run(b, zs):
    dcs = [torch.empty_like(z) for z in zs]
    dvs = [torch.empty_like(z) for z in zs]
    cs, infos = b.gradient(zs, dcs, dvs)
    torch.cuda.synchronize()
    return cs, [i.iters for i in infos], [d.cpu().numpy() for d in dcs]


def _compare(ps, zs, workers=4, **grid_kw):
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32, **grid_kw) for p in ps]
    try:
        with tomo.Batch(workers=workers) as b:
            for g in grids:
                b.append(g)
            launched = _run(b, zs)
            assert b.persistent_info == (0, 0, 0)
            b.set_persistent(True)
            persist = _run(b, zs)
            ctas, phases, runs = b.persistent_info
            b.set_persistent(2)                               # with phase timing
            persist2 = _run(b, zs)
            assert b.persistent_info[2] == runs + 1
            times, launches = b.persistent_phase_times()
            loop_ms = b.phase_times()["loop"]
            assert b.lockstep_runs == 3
        assert len(times) == phases and abs(launches - max(persist2[1])) <= 1
        assert 0.0 < sum(t for _, t in times) <= 1e3 * loop_ms
        assert ctas >= torch.cuda.get_device_properties(0).multi_processor_count
        assert phases > 10 and runs == 1
        for res in (persist, persist2):
            assert res[0] == launched[0]                      # compliances, bitwise
            assert res[1] == launched[1]                      # CG iterations
            assert all(np.array_equal(a, b) for a, b in zip(res[2], launched[2]))
        return launched
    finally:
        for g in grids:
            g.close()


def test_persistent_iteration_equals_launched_lockstep():
    """Grids of 2 to 6 multigrid levels, both problem types: every phase kind except the
    residual replacement."""
    ps = [P.cantilever(4, 2, 2), P.mbb_block(96, 48, 40, volfrac=0.12, rmin=2.5),
          P.cantilever(9, 5, 3), P.mbb_block(33, 17, 9, rmin=1.5), P.cantilever(64, 32, 32)]
    _, iters, _ = _compare(ps, _fields(ps, 900), workers=3)
    assert max(iters) > 10


def test_persistent_iteration_with_residual_replacement():
    """The batched FP64 residual replacement (every 4 iterations) as a phase."""
    ps = P.uneven_cantilever_batch(12, 5)
    _, iters, _ = _compare(ps, _fields(ps, 400), rr_every=4)
    assert max(iters) > 8


def test_persistent_iteration_on_64_uneven_cantilevers():
    ps = P.uneven_cantilever_batch(0, 64)
    zs = [torch.full((p.n_el,), p.volfrac, dtype=torch.float32, device=DEV) for p in ps]
    cs, _, _ = _compare(ps, zs, workers=16)
    assert all(np.isfinite(c) and c > 0 for c in cs)


def test_wait_limit_timeout_is_reported_and_recoverable():
    """A wait limit of 0 ns: the CTAs that reach the first barrier before the last one stop
    the loop with TOMO_ETIMEOUT (no fault, no hang); with the limit back the next call runs
    from scratch and gives the launched loop's result."""
    ps = P.uneven_cantilever_batch(3, 6)
    zs = _fields(ps, 100)
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=4) as b:
            for g in grids:
                b.append(g)
            ref = _run(b, zs)
            b.set_persistent(True)
            with pytest.raises(ValueError):
                b.set_wait_limit(-1)
            b.set_wait_limit(0)
            with pytest.raises(tomo.TomoError) as ei:
                _run(b, zs)
            assert ei.value.status == 5                      # TOMO_ETIMEOUT
            assert b.persistent_info[0] > 0
            x = torch.arange(4, device=DEV, dtype=torch.float32)
            assert float((x * 2).sum()) == 12.0              # the context still works
            b.set_wait_limit(2_000_000_000)
            again = _run(b, zs)
        assert again[0] == ref[0] and again[1] == ref[1]
        assert all(np.array_equal(a, c) for a, c in zip(again[2], ref[2]))
    finally:
        for g in grids:
            g.close()
