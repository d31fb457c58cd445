"""A served request stream through the request loop (``tomo.Server``): Poisson arrivals of
gradient requests on 2n x n x n domains of different sizes (seeded supports, loads and
density fields), device-resident grids, admission under a device-memory budget; reports
p50/p99 latency and throughput, next to serial FP64 GPU gradients on a sample of the same
requests.  --opt-frac mixes in optimisation requests (--opt-iters OC iterations each).
--rate 0 submits every request at once (saturation: the throughput is then the request
loop's capacity).  --max-batch N lets a free worker take up to N queued gradient requests
together as one lockstep batch.

    python -m paper_2104_12282_gb300.serve --requests 1000 --rate 200 --budget-gb 150
"""
from __future__ import annotations

import argparse
import json
import statistics
import sys
import time

import numpy as np

from . import problems as P
from . import tomo


def percentile(xs, q):
    s = sorted(xs)
    return s[min(len(s) - 1, int(round(q * (len(s) - 1))))]


def run_stream(n_requests=1000, rate=200.0, seed=0, workers=16, budget_bytes=150 << 30,
               n_range=(12, 64), serial_sample=12, opt_frac=0.0, opt_iters=10, max_batch=1,
               batch_workers=4):
    reqs = [P.served_request(seed, i, n_range) for i in range(n_requests)]
    if rate > 0:
        gaps = np.random.default_rng([seed, 1]).exponential(1.0 / rate, size=n_requests)
        arrive = np.cumsum(gaps)
    else:   # saturation
        arrive = np.zeros(n_requests)
    # a seeded fraction of the requests are optimisation requests (opt_iters OC iterations)
    is_opt = np.random.default_rng([seed, 2]).random(n_requests) < opt_frac
    lat, qms, lat_opt = [], [], []
    with tomo.Server(workers=workers, budget_bytes=budget_bytes, max_batch=max_batch,
                     batch_workers=batch_workers) as srv:
        t0 = time.perf_counter()
        tickets = []
        for p, ta, o in zip(reqs, arrive, is_opt):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit_optimize(p, opt_iters) if o else srv.submit(p))
        for t, o in zip(tickets, is_opt):
            r, _, _ = srv.wait(t)
            if r.status != 0:
                raise RuntimeError(f"request {t} failed: {r.message.decode()}")
            (lat_opt if o else lat).append(r.queue_ms + r.run_ms)
            qms.append(r.queue_ms)
        wall = time.perf_counter() - t0
        st = srv.stats()
    # serial FP64 GPU gradients on a sample of the same requests (one at a time)
    import torch
    ser = []
    for p in reqs[:serial_sample]:
        with tomo.Grid.from_problem(p, precision=tomo.FP64) as g:
            z = torch.tensor(p.z0, dtype=torch.float64, device="cuda")
            dc = torch.empty_like(z)
            torch.cuda.synchronize()
            t = time.perf_counter()
            g.gradient(z, dc)
            torch.cuda.synchronize()
            ser.append((time.perf_counter() - t) * 1e3)
    return {
        "requests": n_requests, "rate_per_s": rate if rate > 0 else "all at once",
        "workers": workers, "max_batch": max_batch, "batch_workers": batch_workers,
        "budget_gb": budget_bytes / 2 ** 30, "sizes": f"2n x n x n, n ~ U{{{n_range[0]}..{n_range[1]}}}",
        "throughput_per_s": n_requests / wall, "p50_ms": percentile(lat, 0.5),
        "p99_ms": percentile(lat, 0.99), "queue_p99_ms": percentile(qms, 0.99),
        "optimisation_requests": int(is_opt.sum()), "opt_iters": opt_iters if opt_frac > 0 else 0,
        "opt_p50_ms": percentile(lat_opt, 0.5) if lat_opt else None,
        "opt_p99_ms": percentile(lat_opt, 0.99) if lat_opt else None,
        "serial_fp64_ms_mean": statistics.mean(ser), "serial_fp64_per_s": 1e3 / statistics.mean(ser),
        "grids_created": st["grids_created"], "evictions": st["evictions"],
        "lockstep_batches": st["batches"],
        "peak_resident_gb": st["peak_bytes"] / 2 ** 30}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--opt-frac", type=float, default=0.0,
                    help="fraction of the requests that are optimisation requests")
    ap.add_argument("--opt-iters", type=int, default=10,
                    help="OC iterations of an optimisation request")
    ap.add_argument("--max-batch", type=int, default=1,
                    help="lockstep batching: up to this many queued gradient requests per "
                         "batch (1: every request alone on its worker's stream)")
    ap.add_argument("--batch-workers", type=int, default=4)
    a = ap.parse_args(argv)
    out = run_stream(a.requests, a.rate, a.seed, a.workers, int(a.budget_gb * 2 ** 30),
                     opt_frac=a.opt_frac, opt_iters=a.opt_iters, max_batch=a.max_batch,
                     batch_workers=a.batch_workers)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    sys.exit(main())
