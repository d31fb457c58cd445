"""The request loop (tomo_server_*): each result in the mix equals the request's result
alone, under eviction pressure; admission respects the memory budget."""
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


def _alone(p):
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        z = np.asarray(p.z0, np.float32)
        dc = np.empty(p.n_el, np.float32)
        dv = np.empty(p.n_el, np.float32)
        c, info = g.gradient(z, dc, dv)
    return c, dc, dv


def test_results_in_the_mix_equal_results_alone():
    reqs = [P.served_request(3, i, (6, 16)) for i in range(14)]
    # three sessions repeat their problem (device-resident grids reused)
    sessions = [i % 3 if i < 9 else -1 for i in range(len(reqs))]
    for i in range(3, 9):
        reqs[i] = reqs[i % 3]
    budget = 3 * max(tomo.estimate_device_bytes(p) for p in reqs)  # forces evictions
    with tomo.Server(workers=4, budget_bytes=budget) as srv:
        tickets = [srv.submit(p, session=s) for p, s in zip(reqs, sessions)]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["peak_bytes"] <= budget
    assert st["grids_created"] < len(reqs)          # sessions reused their grids
    for p, (r, dc, dv) in zip(reqs, got):
        assert r.status == 0, r.message
        c, dc0, dv0 = _alone(p)
        assert r.compliance == c
        assert np.array_equal(dc, dc0) and np.array_equal(dv, dv0)


def test_eviction_under_a_tight_budget():
    reqs = [P.served_request(4, i, (8, 14)) for i in range(8)]
    budget = max(tomo.estimate_device_bytes(p) for p in reqs) + (1 << 20)
    with tomo.Server(workers=3, budget_bytes=budget) as srv:
        tickets = [srv.submit(p, session=i) for i, p in enumerate(reqs)]
        res = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    assert all(r.status == 0 for r in res)
    assert st["evictions"] >= len(reqs) - 1 and st["peak_bytes"] <= budget


def test_oversized_request_is_rejected():
    p = P.served_request(5, 0, (20, 20))
    with tomo.Server(workers=2, budget_bytes=1 << 20) as srv:
        with pytest.raises(tomo.TomoError):
            srv.submit(p)


def test_estimate_bounds_the_device_memory_of_a_grid():
    for p in (P.cantilever(24, 12, 12), P.mbb_block(33, 17, 9), P.served_request(6, 2, (30, 30))):
        est = tomo.estimate_device_bytes(p)
        with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
            z = np.asarray(p.z0, np.float32)
            dc = np.empty(p.n_el, np.float32)
            dv = np.empty(p.n_el, np.float32)
            g.gradient(z, dc, dv)       # host arrays: staging buffers allocated
            held = g.device_bytes()
        assert held <= est <= 2 * held + (8 << 20), (p.name, held, est)


def test_a_failing_request_does_not_disturb_the_others():
    good = [P.served_request(8, i, (6, 10)) for i in range(4)]
    bad = P.served_request(8, 9, (6, 10))
    bad.nu = 0.7          # rejected at grid creation (Poisson ratio out of range)
    with tomo.Server(workers=2, budget_bytes=1 << 30) as srv:
        tickets = [srv.submit(p) for p in good[:2]] + [srv.submit(bad)] + \
                  [srv.submit(p) for p in good[2:]]
        res = [srv.wait(t) for t in tickets]
    statuses = [r.status for r, _, _ in res]
    assert statuses[2] != 0 and len(res[2][0].message) > 0
    for k, p in zip((0, 1, 3, 4), good):
        r, dc, _ = res[k]
        assert r.status == 0
        c, dc0, _ = _alone(p)
        assert r.compliance == c and np.array_equal(dc, dc0)


def test_optimisation_requests_equal_the_loop_alone():
    """Optimisation requests (OC iterations with warm-started solves on the request's grid)
    give bitwise the final design and last compliance of the same loop run alone; a gradient
    request that follows on the same session grid still gives its cold result alone."""
    ps = [P.served_request(11, i, (6, 12)) for i in range(4)]
    iters = 6
    alone = []
    for p in ps:
        with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
            g.set_warm_start(True)
            z = torch.tensor(np.asarray(p.z0, np.float32), device="cuda")
            dc, dv, zn = torch.empty_like(z), torch.empty_like(z), torch.empty_like(z)
            for _ in range(iters):
                c, info = g.gradient(z, dc, dv)
                g.oc_step(z, dc, dv, p.volfrac, p.move, zn)
                z, zn = zn, z
            torch.cuda.synchronize()
            alone.append((c, info.iters, z.cpu().numpy()))
    with tomo.Server(workers=3, budget_bytes=1 << 30) as srv:
        tickets = [srv.submit_optimize(p, iters, session=(i if i % 2 else -1))
                   for i, p in enumerate(ps)]
        tickets.append(srv.submit(ps[1], session=1))
        res = [srv.wait(t) for t in tickets]
    for (c, it, z), (r, zo, _) in zip(alone, res[:4]):
        assert r.status == 0, r.message
        assert r.compliance == c and r.info.iters == it
        assert np.array_equal(zo, z)
    r, dc, _ = res[4]
    c0, dc0, _ = _alone(ps[1])
    assert r.status == 0 and r.compliance == c0 and np.array_equal(dc, dc0)


def test_bad_optimisation_requests_are_rejected():
    p = P.served_request(12, 0, (6, 8))
    with tomo.Server(workers=1, budget_bytes=1 << 30) as srv:
        for kw in (dict(iters=0), dict(iters=3, volfrac=0.0), dict(iters=3, move=0.0)):
            with pytest.raises(tomo.TomoError):
                srv.submit_optimize(p, **kw)


def _close(c, dc, c0, dc0):
    den = np.maximum(np.abs(dc0), 1e-3 * np.abs(dc0).max())
    return abs(c / c0 - 1.0) <= 1e-5 and float(np.max(np.abs(dc - dc0) / den)) <= 1e-4


def test_lockstep_batched_requests_agree_with_results_alone():
    """With lockstep batching the queued gradient requests a free worker takes run as one
    tomo_batch; each result agrees with the request alone to the solver's tolerance, a
    repeated session reuses its grid, and a request that fails at grid creation fails alone."""
    reqs = [P.served_request(13, i, (6, 14)) for i in range(12)]
    reqs[7] = reqs[2]
    bad = P.served_request(13, 40, (6, 10))
    bad.nu = 0.7                                 # rejected at grid creation
    sessions = [-1] * 12
    sessions[2] = sessions[7] = 5
    with tomo.Server(workers=2, budget_bytes=1 << 30, max_batch=8, batch_workers=2) as srv:
        tickets = [srv.submit(p, session=s) for p, s in zip(reqs, sessions)]
        tb = srv.submit(bad)
        got = [srv.wait(t) for t in tickets]
        rb = srv.wait(tb)[0]
        st = srv.stats()
    assert st["completed"] == len(reqs) + 1 and st["batches"] >= 1
    assert rb.status != 0 and len(rb.message) > 0
    for p, (r, dc, dv) in zip(reqs, got):
        assert r.status == 0, r.message
        c0, dc0, dv0 = _alone(p)
        assert _close(r.compliance, dc, c0, dc0), p.dims
        assert np.array_equal(dv, dv0)           # dV/dz involves no solve
