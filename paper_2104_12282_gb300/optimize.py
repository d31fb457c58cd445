"""Optimisation runs on the GPU through the C ABI: Algorithm 1 with the exact gradient on
every iteration (the optimiser the paper compares against), with the two-scale coarse
step at the top of each iteration when a block size is given (coarse-grain z, solve the
coarse state K_C(z_C) u_C = f_C).  The synthetic-gradient model of Algorithm 1 is not
part of this package.

    python -m paper_2104_12282_gb300.optimize --mesh 1 --iters 200 --block 5

runs the cantilever of §IV on the Table 1 meshes (domain 2 x 1 x 1, element edge 1/ny,
filter radius 0.08 in domain units, volume fraction 0.12) and prints one JSON line per
iteration and a summary line.  p = 3, E0 = 1, Emin = 1e-9 and the OC constants (move 0.2,
eta 1/2) are readings: the paper does not state them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import problems as P
from . import tomo

MESHES = {1: (70, 35, 35), 2: (100, 50, 50), 3: (180, 90, 90)}


def paper_cantilever(mesh: int, volfrac: float = 0.12, radius: float = 0.08) -> P.Problem:
    """Cantilever Mesh 1-3 of Table 1 in domain units: h = 1/ny, rmin = radius / h."""
    nx, ny, nz = MESHES[mesh]
    h = 1.0 / ny
    return P.cantilever(nx, ny, nz, h=h, volfrac=volfrac, rmin=radius / h)


def save_checkpoint(path: str, k: int, z, hist, smoother) -> None:
    """State of an OC run after its iteration k-1 (the design z, the history so far and the
    smoother setting (fine, coarse, ratio[, bound, W-cycle mask])), written atomically
    (temporary file, then rename)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, next_it=np.int64(k), z=np.asarray(z),
             smoother=np.asarray(smoother, np.float64),
             hist=np.frombuffer(json.dumps(hist).encode(), dtype=np.uint8))
    os.replace(tmp, path)


def load_checkpoint(path: str):
    """(next iteration, z, history, smoother) from save_checkpoint; the smoother as
    (fine, coarse[, ratio, bound, W-cycle mask])."""
    with np.load(path) as f:
        sm = [float(v) for v in f["smoother"]]
        smoother = tuple([int(sm[0]), int(sm[1])] + sm[2:4] + [int(v) for v in sm[4:5]])
        return (int(f["next_it"]), f["z"], json.loads(bytes(f["hist"]).decode()), smoother)


def smoother_state(g) -> tuple:
    """(fine, coarse, ratio, bound, W-cycle mask): the grid's full smoother setting."""
    fine, coarse, ratio = g.smoother()
    return (fine, coarse, ratio, g.smoother_bound()[0], g.cycle())


def set_smoother_state(g, sm) -> None:
    g.set_smoother(sm[0], sm[1], *sm[2:3])
    if len(sm) > 3:
        g.set_smoother_bound(sm[3])
        g.set_cycle(sm[4])


def run(problem: P.Problem, iters: int, *, block: int = 0, precision: int = tomo.FP32,
        rtol: float = 1e-6, warm: bool = True, maxit: int = 5000, z0=None, callback=None,
        autotune_every: int = 0, tune: str = "online", checkpoint: str | None = None,
        checkpoint_every: int = 0, resume: bool = False):
    """Exact-gradient OC loop on the GPU.  Returns (z, history); history holds one dict per
    iteration: compliance, design change, CG iterations, wall time of the gradient and of
    the coarse step (ms), and the smoother (fine, coarse degrees) the gradient used.
    autotune_every > 0: the smoother is re-chosen at iterations autotune_every,
    2 autotune_every, ... (the design drifts from the smooth start towards near 0/1
    densities, which favour other smoother degrees).  tune "offline": the library's
    autotuner times extra solves of the current design (not counted in `ms`); "online": the
    next gradients of the run itself try the candidates one each, then the fastest is kept
    (no extra solves; the trial gradients are real iterations of the run).

    checkpoint: a file that receives the run's state every checkpoint_every iterations and
    at the end; resume: continue from that file's state (its design, history and smoother)
    up to iteration `iters`.  The first gradient after a resume starts its solve from zero
    (the displacement is not stored), so the resumed run follows the uninterrupted one to
    the solver's tolerance, not bitwise."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    dt = torch.float32 if precision == tomo.FP32 else torch.float64
    z = torch.tensor(np.asarray(problem.z0 if z0 is None else z0), dtype=dt, device=dev)
    zn = torch.empty_like(z)
    dc = torch.empty_like(z)
    dv = torch.empty_like(z)
    hist = []
    start = 0
    resumed_smoother = None
    if resume:
        start, zr, hist, resumed_smoother = load_checkpoint(checkpoint)
        z = torch.tensor(zr, dtype=dt, device=dev)
        zn = torch.empty_like(z)
    cands = [(2, 2), (2, 3), (2, 4), (1, 3), (1, 4), (1, 6)]
    trial = []      # online tuning: (candidate, ms) of the trial gradients so far
    with tomo.Grid.from_problem(problem, precision=precision, rtol=rtol, maxit=maxit) as g:
        g.set_warm_start(warm)
        if resumed_smoother is not None:
            set_smoother_state(g, resumed_smoother)
        gc = None
        if block:
            q = P.coarse_problem(problem, block)
            gc = tomo.Grid.from_problem(q, precision=precision, rtol=rtol, maxit=maxit)
            gc.set_warm_start(warm)
            zc = torch.empty(q.n_el, dtype=dt, device=dev)
            uc = torch.zeros(q.dims.n_dof, dtype=dt, device=dev)
        try:
            for k in range(start, iters):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                coarse = None
                if gc is not None:   # Algorithm 1: coarse-grain z, solve the coarse state
                    g.coarse_grain(z, block, zc)
                    ci = gc.solve(zc, uc)
                    coarse = ci.iters
                tuned = None
                if autotune_every > 0 and k > 0 and k % autotune_every == 0:
                    if tune == "offline":
                        tuned, _ = g.autotune(z, reps=1)
                    else:
                        trial = [None] * len(cands)
                if trial and None in trial:     # online: this gradient tries a candidate
                    g.set_smoother(*cands[trial.index(None)])
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                c, info = g.gradient(z, dc, dv)
                change = g.oc_step(z, dc, dv, problem.volfrac, problem.move, zn)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                if trial and None in trial:
                    trial[trial.index(None)] = (t2 - t1)
                    if None not in trial:      # all tried: keep the fastest
                        tuned = cands[int(np.argmin(trial))]
                        g.set_smoother(*tuned)
                        trial = []
                rec = dict(it=k, c=c, change=change, cg_iters=info.iters,
                           ms=(t2 - t1) * 1e3, coarse_ms=(t1 - t0) * 1e3,
                           coarse_cg_iters=coarse, smoother=list(g.smoother()[:2]),
                           tuned=tuned is not None)
                hist.append(rec)
                if callback:
                    callback(rec)
                z, zn = zn, z
                if checkpoint and ((checkpoint_every > 0 and (k + 1) % checkpoint_every == 0)
                                   or k + 1 == iters):
                    save_checkpoint(checkpoint, k + 1, z.cpu().numpy(), hist,
                                    smoother_state(g))
        finally:
            if gc is not None:
                gc.close()
    return z, hist


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--mesh", type=int, choices=sorted(MESHES), default=1)
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--block", type=int, default=5, help="two-scale block size N_B (0: off)")
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--cold", action="store_true", help="start every solve from zero")
    ap.add_argument("--quiet", action="store_true")
    ap.add_argument("--autotune-every", type=int, default=0,
                    help="re-choose the smoother every N iterations (0: off)")
    ap.add_argument("--tune", choices=("online", "offline"), default="online",
                    help="online: try the candidates on the run's own gradients; offline: "
                         "the library autotuner's extra solves")
    ap.add_argument("--checkpoint", default=None, help="state file (written every "
                    "--checkpoint-every iterations and at the end)")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
    a = ap.parse_args(argv)
    p = paper_cantilever(a.mesh)
    prec = tomo.FP64 if a.fp64 else tomo.FP32

    def show(rec):
        if not a.quiet:
            print(json.dumps(rec), flush=True)

    t = time.perf_counter()
    _, hist = run(p, a.iters, block=a.block, precision=prec, warm=not a.cold, callback=show,
                  autotune_every=a.autotune_every, tune=a.tune, checkpoint=a.checkpoint,
                  checkpoint_every=a.checkpoint_every, resume=a.resume)
    wall = time.perf_counter() - t
    d = p.dims
    print(json.dumps({"mesh": a.mesh, "dims": [d.nx, d.ny, d.nz], "h": p.h, "rmin": p.rmin,
                      "block": a.block, "iters": a.iters, "final_c": hist[-1]["c"],
                      "wall_s": wall, "cg_iters_total": sum(r["cg_iters"] for r in hist),
                      "precision": "fp64" if a.fp64 else "fp32-mixed",
                      "warm_start": not a.cold, "autotune_every": a.autotune_every,
                      "tune": a.tune if a.autotune_every else None,
                      "smoother_final": hist[-1]["smoother"],
                      "gradient_s": sum(r["ms"] for r in hist) / 1e3}), flush=True)


if __name__ == "__main__":
    sys.exit(main())
