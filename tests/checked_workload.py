"""Workload run against one build of the library (the regular or, with TOMO_LIB=checked,
the bounds-checked one) by tests/test_gpu_checked.py: products, gradients and OC steps on
small and odd grids in both precisions, a wide filter, the general adjoint, the two-scale
coarse-graining, lockstep batches (8- and 4-row tiles, the persistent iteration), a W-cycle,
the coarse tail in one cluster launch and a served request.  Prints one JSON object: the results and the check report."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from paper_2104_12282_gb300 import problems as P  # noqa: E402
from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def t(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device=DEV)


def run():
    out = {}
    for dims in [(1, 1, 1), (2, 1, 1), (3, 2, 5), (17, 9, 5), (33, 17, 9), (7, 31, 4)]:
        for kind in ("cantilever", "mbb"):
            p = P.cantilever(*dims) if kind == "cantilever" else P.mbb_block(*dims, rmin=1.5)
            for prec, dt in ((tomo.FP32, torch.float32), (tomo.FP64, torch.float64)):
                key = "%s_%dx%dx%d_%s" % (kind, *dims, "f32" if prec == tomo.FP32 else "f64")
                z = t(P.random_field(p.dims, 1, 0.05, 1.0), dt)
                x = t(P.random_nodal(p.dims, 2), dt)
                with tomo.Grid.from_problem(p, precision=prec) as g:
                    y = torch.empty(p.dims.n_dof, dtype=dt, device=DEV)
                    g.apply_stiffness(z, x, y)
                    dc, dv, zn = (torch.empty_like(z) for _ in range(3))
                    c, info = g.gradient(z, dc, dv)
                    g.oc_step(z, dc, dv, p.volfrac, p.move, zn)
                    torch.cuda.synchronize()
                    out[key] = [float(y.abs().sum()), c, info.iters, float(dc.sum()),
                                float(zn.sum())]
    # wide filter, adjoint, two-scale coarse-graining
    p = P.cantilever(24, 12, 12, rmin=5.0)
    z = t(P.random_field(p.dims, 3, 0.05, 1.0))
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        dc = torch.empty_like(z)
        c, _ = g.gradient(z, dc)
        l = t(P.random_nodal(p.dims, 4))
        dj = torch.empty_like(z)
        J, _, _ = g.adjoint_gradient(z, l, dj)
        cx, cy, cz = tomo.coarse_dims(24, 12, 12, 4)
        zc = torch.empty(cx * cy * cz, dtype=torch.float32, device=DEV)
        g.coarse_grain(z, 4, zc)
        g.set_cycle(2)
        c2, _ = g.gradient(z, dc)
        g.set_cycle(0)
        g.set_coarse_tail(True)
        c3, _ = g.gradient(z, dc)
        torch.cuda.synchronize()
        out["wide_adjoint_twoscale_w_tail"] = [c, J, float(dj.sum()), float(zc.sum()), c2, c3]
    # lockstep batches
    ps = P.uneven_cantilever_batch(5, 6)
    zs = [t(P.random_field(q.dims, 10 + i, 0.05, 1.0)) for i, q in enumerate(ps)]
    grids = [tomo.Grid.from_problem(q, precision=tomo.FP32, rr_every=4) for q in ps]
    try:
        with tomo.Batch(workers=2) as b:
            for g in grids:
                b.append(g)
            for rows, persist in ((8, False), (4, False), (8, True)):
                b.set_tiles(rows, 4)
                b.set_persistent(persist)
                dcs = [torch.empty_like(zz) for zz in zs]
                cs, _ = b.gradient(zs, dcs)
                torch.cuda.synchronize()
                out["batch_%d_%d" % (rows, int(persist))] = list(cs)
    finally:
        for g in grids:
            g.close()
    # a served request
    with tomo.Server(workers=1, budget_bytes=1 << 30) as srv:
        r, dcs, _ = srv.wait(srv.submit(P.served_request(2, 0, (6, 10))))
        out["served"] = [r.status, r.compliance, float(np.sum(dcs))]
    checked, word = tomo.check_report()
    return {"checked": checked, "word": word, "results": out}


if __name__ == "__main__":
    print(json.dumps(run()))
