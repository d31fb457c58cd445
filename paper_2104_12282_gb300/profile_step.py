"""The benchmark step (gradient + OC update on the 192x96x76 MBB-type block, bumpy field)
with every kernel issued from the host, for profilers: ncu does not profile kernel nodes
of graphs with conditional nodes, so the CG loop normally hidden in such a graph is issued
as separate launches here (bitwise the same results).  Single host thread, one grid.

    python -m paper_2104_12282_gb300.profile_step --steps 2 [--degrees 2,2 --bound-scale 0.68]
"""
from __future__ import annotations

import argparse
import sys

from . import problems as P
from . import tomo


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--degrees", default="2,2", help="fine,coarse Chebyshev degrees")
    ap.add_argument("--bound-scale", type=float, default=1.0,
                    help="smoothing-interval bound as a fraction of the element bound")
    ap.add_argument("--ratio", type=float, default=20.0, help="smoothing-interval ratio")
    a = ap.parse_args(argv)
    import torch

    p = P.mbb_192x96x76(a.seed)
    prec = tomo.FP64 if a.fp64 else tomo.FP32
    dt = torch.float64 if a.fp64 else torch.float32
    dev = torch.device("cuda", 0)
    z = torch.tensor(P.bumpy_field(p.dims, a.seed), dtype=dt, device=dev)
    dc, dv, zn = torch.empty_like(z), torch.empty_like(z), torch.empty_like(z)
    with tomo.Grid.from_problem(p, precision=prec, maxit=5000) as g:
        fine, coarse = (int(v) for v in a.degrees.split(","))
        g.set_smoother(fine, coarse, a.ratio)
        g.set_smoother_bound(a.bound_scale * g.smoother_bound()[1])
        g.profile_enable(True)   # host-issued CG iterations, events around the products
        for _ in range(a.steps):
            c, info = g.gradient(z, dc, dv)
            g.oc_step(z, dc, dv, p.volfrac, p.move, zn)
        torch.cuda.synchronize()
        n, ms, byt = g.profile_read()
        g.profile_enable(False)
    print(f"compliance {c:.9g}, CG iterations {info.iters}, fine-level product launches {n}, "
          f"{ms / max(n, 1) * 1e3:.1f} us each", flush=True)


if __name__ == "__main__":
    sys.exit(main())
