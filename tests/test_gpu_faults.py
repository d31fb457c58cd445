"""Host-side fault injection (tomo_inject_fault / TOMO_FAULT): each error path returns its
status and message, the handle stays usable and the next call gives the clean result.  No
GPU fault is made: the host reports an error in place of the real call's result (a device
allocation, a stream synchronisation after the real one, a CG-loop graph launch that is
not made), writes a NaN modulus into the material (a valid value the solve must report),
or delays a served request on the host."""
import os
import subprocess
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
ENOMEM, ENAN, ECUDA = 2, 4, 6


def _field(p, seed):
    return torch.tensor(P.random_field(p.dims, seed, 0.05, 1.0), dtype=torch.float32,
                        device=DEV)


def _grad(g, z):
    dc = torch.empty_like(z)
    c, info = g.gradient(z, dc)
    torch.cuda.synchronize()
    return c, info.iters, dc.cpu().numpy()


def test_unknown_sites_and_negative_counts_are_rejected():
    for site, n in (("nope", 1), ("alloc", -1), ("", 1)):
        with pytest.raises(tomo.TomoError):
            tomo.inject_fault(site, n)
    tomo.inject_fault("alloc", 0)        # disarm: a no-op here


def test_injected_allocation_failure_at_grid_creation():
    p = P.cantilever(12, 6, 6)
    tomo.inject_fault("alloc", 3)
    with pytest.raises(tomo.TomoError) as ei:
        tomo.Grid.from_problem(p, precision=tomo.FP32)
    assert ei.value.status == ENOMEM and "injected" in str(ei.value)
    z = _field(p, 1)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        c, it, dc = _grad(g, z)
    assert np.isfinite(c) and c > 0 and it > 0


def test_injected_sync_and_graph_failures_leave_the_grid_usable():
    p = P.mbb_block(24, 12, 10, rmin=1.5)
    z = _field(p, 2)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        ref = _grad(g, z)
        for site in ("sync", "graph"):
            tomo.inject_fault(site, 1)
            with pytest.raises(tomo.TomoError) as ei:
                _grad(g, z)
            assert ei.value.status == ECUDA and "injected" in str(ei.value)
            again = _grad(g, z)
            assert again[0] == ref[0] and again[1] == ref[1]
            assert np.array_equal(again[2], ref[2])


def test_injected_nan_modulus_is_reported_and_the_grid_recovers():
    p = P.cantilever(16, 8, 8)
    z = _field(p, 3)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        ref = _grad(g, z)
        tomo.inject_fault("nan_input", 1)
        with pytest.raises(tomo.TomoError) as ei:
            _grad(g, z)
        assert ei.value.status == ENAN
        again = _grad(g, z)
    assert again[0] == ref[0] and again[1] == ref[1] and np.array_equal(again[2], ref[2])


def test_a_slow_request_does_not_hold_up_the_others():
    reqs = [P.served_request(9, i, (6, 10)) for i in range(4)]
    with tomo.Server(workers=2, budget_bytes=1 << 30) as srv:
        tomo.inject_fault("slow_request", 1)
        tickets = [srv.submit(p) for p in reqs]
        res = [srv.wait(t) for t in tickets]
    assert all(r.status == 0 for r, _, _ in res)
    slow = [r for r, _, _ in res if r.run_ms >= 200.0]
    fast = [r for r, _, _ in res if r.run_ms < 200.0]
    assert len(slow) == 1 and len(fast) == 3
    assert max(r.queue_ms + r.run_ms for r in fast) < slow[0].queue_ms + slow[0].run_ms


def test_injected_graph_failure_in_a_lockstep_batch():
    ps = P.uneven_cantilever_batch(5, 4)
    zs = [_field(p, 10 + i) for i, p in enumerate(ps)]
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        with tomo.Batch(workers=2) as b:
            for g in grids:
                b.append(g)

            def run():
                dcs = [torch.empty_like(z) for z in zs]
                cs, infos = b.gradient(zs, dcs)
                torch.cuda.synchronize()
                return cs, [i.iters for i in infos], [d.cpu().numpy() for d in dcs]

            ref = run()
            tomo.inject_fault("graph", 1)
            with pytest.raises(tomo.TomoError) as ei:
                run()
            assert ei.value.status == ECUDA and "injected" in str(ei.value)
            again = run()
        assert again[0] == ref[0] and again[1] == ref[1]
        assert all(np.array_equal(a, r) for a, r in zip(again[2], ref[2]))
    finally:
        for g in grids:
            g.close()


def test_a_request_with_an_injected_failure_fails_alone():
    reqs = [P.served_request(8, i, (6, 10)) for i in range(3)]
    with tomo.Server(workers=1, budget_bytes=1 << 30) as srv:
        tomo.inject_fault("alloc", 1)      # the first grid the loop creates
        tickets = [srv.submit(p) for p in reqs]
        res = [srv.wait(t) for t in tickets]
    st = [r.status for r, _, _ in res]
    assert st[0] == ENOMEM and b"injected" in res[0][0].message
    for p, (r, dc, _) in zip(reqs[1:], res[1:]):
        assert r.status == 0
        with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
            dc0 = np.empty(p.n_el, np.float32)
            c0, _ = g.gradient(np.asarray(p.z0, np.float32), dc0, np.empty_like(dc0))
        assert r.compliance == c0 and np.array_equal(dc, dc0)


def test_the_environment_arms_a_site():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2104_12282_gb300 import problems as P, tomo\n"
            "try:\n"
            "    tomo.Grid.from_problem(P.cantilever(8, 4, 4), precision=tomo.FP32)\n"
            "    print('created')\n"
            "except tomo.TomoError as e:\n"
            "    print('status', e.status)\n") % ROOT
    env = dict(os.environ, TOMO_FAULT="sync:99,alloc:1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip().splitlines()[-1] == "status %d" % ENOMEM
