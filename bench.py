#!/usr/bin/env python
"""Exact-gradient throughput on GB300: gradient evaluations/s on the 192x96x76 MBB-type
block (1,400,832 voxels, 4,324,551 DOFs), mixed FP32/FP64 path against the all-FP64 GPU
path of the same algorithm, with compliance error and p50/p99 step latency.

One step = the whole hot path on one design field: density filter and SIMP material,
multigrid level setup, GMG-preconditioned CG from a zero start to ||r|| <= 1e-6 ||f||,
compliance and sensitivity, filter adjoint of the sensitivity and of the volume, and one
optimality-criteria update (tomo_gradient + tomo_oc_step).  Inputs are resident on the
device when the timed region starts; L2 is flushed (256 MiB write) between steps, outside
the timed events.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): one independent replica per GPU ("replicas only": the path has no
exchange step), value = all steps of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("grad evals/s @1.4M voxels, mixed vs FP64 GPU at ≤1e-5 compliance err; p99 ms")
UNIT = "grad evals/s"
WORKLOAD = "mbb_block 192x96x76 (1,400,832 voxels, 4,324,551 DOFs), bumpy density field"
SAMPLE_DIMS = (48, 24, 19)   # CPU oracle sample: same recipe on 1/64 of the voxels
SMALL_SAMPLE_DIMS = (24, 12, 10)  # reference arm with many steps: ~1/8 of that
REF_STEPS_FULL_SAMPLE = 40  # above this many warm-up + timed steps, the small sample


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--seed", type=int, default=0)
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------------
# Replicas: one process per GPU, no exchange on the data path; the process group only
# brackets the timed region (barrier) and takes the slowest rank's time.
# ---------------------------------------------------------------------------------------
def init_ranks(backend):
    """torch.distributed module with the default group initialised, or None at N = 1."""
    world, _, _ = dist_env()
    if world == 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(dist, x, device=None):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps_per_rank, slowest_ms):
    """Units processed by all ranks divided by the slowest rank's time (units/s)."""
    return world * steps_per_rank / (slowest_ms * 1e-3)


# ---------------------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------
def oracle_sample(seed, dims=SAMPLE_DIMS):
    """One exact-gradient evaluation plus OC step by the FP64 oracle on a sample box of the
    benchmark recipe (Jacobi-PCG to 1e-6, the paper's standard solver form).  Returns
    (seconds, cores, voxels)."""
    from oracle import topopt
    from paper_2104_12282_gb300 import problems as P
    p = P.mbb_block(*dims, volfrac=0.12, rmin=2.5)
    p.z0 = P.bumpy_field(p.dims, seed)
    m = topopt.Model(p)
    t0 = time.perf_counter()
    c0 = os.times()
    g = m.gradient(p.z0, "pcg", tol=1e-6)
    m.oc_step(p.z0, g["dcdz"], g["dvdz"])
    dt = time.perf_counter() - t0
    c1 = os.times()
    cpu = (c1.user + c1.system) - (c0.user + c0.system)
    return dt, max(1, round(cpu / dt)), p.n_el


def cpu_baseline(seed, reps=3):
    from paper_2104_12282_gb300 import problems as P
    full = P.GridDims(192, 96, 76).n_el
    ts, cores = [], []
    n_sample = None
    for r in range(reps):
        dt, c, n_sample = oracle_sample(seed + r)
        ts.append(dt)
        cores.append(c)
    t = statistics.mean(ts)
    value = (n_sample / full) / t
    return {"value": value, "unit": UNIT, "cores": int(max(cores)), "kind": "oracle",
            "cores_available": os.cpu_count(),
            "sample": (f"FP64 oracle (numpy/scipy): filter, Jacobi-PCG to 1e-6, sensitivity, "
                       f"filter adjoint, OC on the same recipe at {SAMPLE_DIMS[0]}x"
                       f"{SAMPLE_DIMS[1]}x{SAMPLE_DIMS[2]} ({n_sample} voxels), mean of {reps} "
                       f"runs ({t:.2f} s each), scaled to 1,400,832 voxels by element count "
                       f"(flatters the CPU: Jacobi-PCG iteration counts grow with the grid)")}


def cpu_baseline_one_core(seed):
    """The same oracle sample with every BLAS/OpenMP pool held to one thread (a child
    process, so the setting takes effect before numpy loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%d)))" % (ROOT, seed))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0:
        return {"unavailable": r.stderr.strip().splitlines()[-1] if r.stderr else "failed"}
    dt, cores, n_sample = json.loads(r.stdout.strip().splitlines()[-1])
    from paper_2104_12282_gb300 import problems as P
    full = P.GridDims(192, 96, 76).n_el
    return {"value": (n_sample / full) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"as cpu_baseline, one run with thread pools held to 1 ({dt:.2f} s)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    ts = []
    cores = 1
    n_sample = None
    from paper_2104_12282_gb300 import problems as P
    full = P.GridDims(192, 96, 76).n_el
    # each step is a bounded sample: the 1/64 box (~2-5 s of CPU work), or the ~1/490 box
    # when that many steps would not end within a few minutes
    dims = SAMPLE_DIMS if args.warmup + args.steps <= REF_STEPS_FULL_SAMPLE else SMALL_SAMPLE_DIMS
    for s in range(args.warmup + args.steps):
        dt, c, n_sample = oracle_sample(args.seed + s, dims)
        if s >= args.warmup:
            ts.append(dt)
            cores = max(cores, c)
    mean = statistics.mean(ts)
    value = (n_sample / full) / mean
    sample = (f"each step is one FP64 oracle gradient+OC on the {dims[0]}x{dims[1]}x{dims[2]} "
              f"box of the same recipe ({n_sample} voxels); ms_per_step is that step's "
              f"measured time; value is the full-grid rate at the sample's time per voxel "
              f"(sample voxels / 1,400,832 / seconds per step)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": sample, "solver": "Jacobi-PCG 1e-6",
                      "sample_dims": list(dims), "sample_voxels": n_sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
class ClockSampler:
    """SM clocks and throttle reasons sampled by nvidia-smi every 50 ms (200 ms if nvidia-smi
    exits without a row at the shorter interval).

    Entering starts the sampler and waits (at most ``wait_s``) for its first row, so that
    nvidia-smi's own start-up is over before the timed region; enter before the warm-up
    steps.  ``mark()`` at the start of the timed region drops the rows taken before it (an
    idle GPU there reads a low clock); at exit, if no row has arrived since the mark, the
    sampler waits up to two intervals for one."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVALS_MS = (50, 200)

    def __init__(self, index, exe="nvidia-smi", wait_s=5.0):
        self.index = index
        self.exe = exe
        self.wait_s = wait_s
        self.proc = None
        self.thread = None
        self._rows = []
        self.rows = []
        self.first = 0
        self.interval_ms = None

    def _start(self, ms):
        proc = subprocess.Popen(
            [self.exe, "-i", str(self.index), f"--query-gpu={self.FIELDS}",
             "--format=csv,noheader,nounits", "-lms", str(ms)],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        rows = []
        seen = threading.Event()

        def pump():
            for line in proc.stdout:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
                    seen.set()
            seen.set()

        t = threading.Thread(target=pump, daemon=True)
        t.start()
        seen.wait(timeout=self.wait_s)
        return proc, rows, t

    def __enter__(self):
        for ms in self.INTERVALS_MS:
            try:
                proc, rows, t = self._start(ms)
            except (FileNotFoundError, OSError):
                return self
            if rows or proc.poll() is None:
                self.proc, self._rows, self.thread, self.interval_ms = proc, rows, t, ms
                return self
            proc.wait()
            t.join(timeout=5)
        return self

    def mark(self):
        """The timed region starts now."""
        self.first = len(self._rows)

    def __exit__(self, *a):
        if self.proc is None:
            return
        deadline = time.perf_counter() + 2 * self.interval_ms / 1000.0
        while (len(self._rows) <= self.first and self.proc.poll() is None
               and time.perf_counter() < deadline):
            time.sleep(0.005)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.thread.join(timeout=5)
        self.rows = list(self._rows[self.first:])

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows), "interval_ms": self.interval_ms}


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def march2_source_digest():
    """sha256 over the fused FP32 kernel's sources: its launch file, then its body."""
    h = hashlib.sha256()
    for f in ("matvec2.cu", "march2_body.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2104_12282_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def march_traffic():
    """Average DRAM bytes per level-0 launch of the fused FP32 product/smoother kernel, from
    the committed ncu summary; valid only while the kernel source is unchanged."""
    summ = os.path.join(ROOT, "profiles", "k_march2_traffic.json")
    try:
        digest = march2_source_digest()
        rec = json.load(open(summ))
        if rec.get("source_sha256") == digest:
            return float(rec["dram_bytes_per_level0_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


GOLDEN = os.path.join(ROOT, "tests", "golden", "fullsize_mbb_192x96x76_seed0.txt")


def oracle_golden():
    """The FP64 oracle's exact gradient of the benchmark field (seed 0), as stored by
    tests/golden/make_fullsize_goldens.py: (scalars, element indices, dc/dz), or None."""
    try:
        scal, idx, val = {}, [], []
        with open(GOLDEN) as fh:
            for line in fh:
                if line.startswith("#") or not line.strip():
                    continue
                a, b = line.split()
                if a.isdigit():
                    idx.append(int(a))
                    val.append(float(b))
                else:
                    scal[a] = float(b)
        return scal, idx, val
    except (OSError, ValueError):
        return None


def extras(args, dev, stream):
    """Side measurements on one GPU, after the timed steps: an OC-evolved field on the
    benchmark grid (near 0/1 densities raise CG iteration counts), the two-scale step of
    Algorithm 1 at N_B = 4, and the batch of 64 uneven cantilevers."""
    import torch

    from paper_2104_12282_gb300 import problems as P
    from paper_2104_12282_gb300 import tomo

    def timed(fn, reps):
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.mean(ms), r

    out = {}
    p = P.mbb_192x96x76(args.seed)
    kw = dict(precision=tomo.FP32, maxit=5000, stream=stream.cuda_stream)
    with tomo.Grid.from_problem(p, **kw) as g:
        z = torch.full((p.n_el,), p.volfrac, dtype=torch.float32, device=dev)
        zn, dc, dv = torch.empty_like(z), torch.empty_like(z), torch.empty_like(z)
        g.set_warm_start(True)
        t0 = time.perf_counter()
        warm_its = []
        for _ in range(50):
            c, info = g.gradient(z, dc, dv)
            warm_its.append(info.iters)
            g.oc_step(z, dc, dv, p.volfrac, p.move, zn)
            z, zn = zn, z
        torch.cuda.synchronize()
        loop_s = time.perf_counter() - t0
        g.set_warm_start(False)
        g.gradient(z, dc, dv)
        ms, (c, info) = timed(lambda: g.gradient(z, dc, dv), 3)
        best, _ = g.autotune(z)    # smoother autotuner on the evolved design
        g.gradient(z, dc, dv)
        ms_t, (c_t, info_t) = timed(lambda: g.gradient(z, dc, dv), 3)
        g.set_smoother(2, 2, 20.0)
        g.set_smoother_bound(0.0)
        g.set_cycle(0)
        out["evolved_field"] = {
            "recipe": "50 OC iterations from the uniform start (volfrac 0.12), warm-started "
                      "solves; then cold-start gradients on that design",
            "cold_ms_per_grad": ms, "cold_cg_iters": info.iters,
            "oc_loop_s_50_iters": loop_s, "warm_cg_iters_last": warm_its[-1],
            "warm_cg_iters_mean": statistics.mean(warm_its),
            "autotuned": {"fine_degree": best[0], "coarse_degree": best[1],
                          "smoothing_bound": best[2], "w_cycle_levels": best[3],
                          "interval_ratio": best[4],
                          "cold_ms_per_grad": ms_t, "cold_cg_iters": info_t.iters}}
        # two-scale step of Algorithm 1 at N_B = 4 on the bumpy field
        nb = 4
        q = P.coarse_problem(p, nb)
        zb = torch.tensor(P.bumpy_field(p.dims, args.seed), dtype=torch.float32, device=dev)
        with tomo.Grid.from_problem(q, **kw) as gc:
            zc = torch.empty(q.n_el, dtype=torch.float32, device=dev)
            uc = torch.zeros(q.dims.n_dof, dtype=torch.float32, device=dev)

            def step():
                g.coarse_grain(zb, nb, zc)
                uc.zero_()   # tomo_solve starts from u: cold start, as the fine gradient
                return gc.solve(zc, uc)
            step()
            ms, info = timed(step, 3)
            out["two_scale"] = {"block": nb, "coarse_dims": [q.dims.nx, q.dims.ny, q.dims.nz],
                                "coarse_dofs": q.dims.n_dof, "ms": ms,
                                "coarse_cg_iters": info.iters,
                                "step": "tomo_coarse_grain + tomo_solve on the coarse grid"}
    # batch of 64 uneven cantilevers
    ps = P.uneven_cantilever_batch(args.seed, 64)
    grids = [tomo.Grid.from_problem(q, **kw) for q in ps]
    try:
        zs = [torch.tensor(P.random_field(q.dims, args.seed + i, 0.05, 1.0), dtype=torch.float32,
                           device=dev) for i, q in enumerate(ps)]
        dcs = [torch.empty_like(t) for t in zs]
        loops = {}
        with tomo.Batch(workers=8) as b:
            for gg in grids:
                b.append(gg)
            # product tiles (rows per CTA, waves) chosen by the library's tile autotuner on
            # other fields of the same recipe, untimed
            zt = [torch.tensor(P.random_field(q.dims, args.seed + 100 + i, 0.05, 1.0),
                               dtype=torch.float32, device=dev) for i, q in enumerate(ps)]
            tiles, tile_rows = b.autotune_tiles(zt, dcs, reps=2)
            del zt
            # the lockstep loop with one launch per phase at the tuned tiles, then with one
            # cooperative launch per CG iteration (tomo_batch_set_persistent), which runs
            # 8-row tiles
            for persist in (False, True):
                b.set_persistent(persist)
                b.set_tiles(*(tiles if not persist else (8, tiles[1])))
                b.gradient(zs, dcs)
                torch.cuda.synchronize()
                # each call returns once its compliances are on the host: time 10 calls one
                # by one and keep the median (a host hiccup in one call moved a 3-call mean
                # by 5 %)
                calls = []
                for _ in range(10):
                    t0 = time.perf_counter()
                    cs, infos = b.gradient(zs, dcs)
                    torch.cuda.synchronize()
                    calls.append(time.perf_counter() - t0)
                loops[persist] = (statistics.median(calls), b.phase_times()["loop"],
                                  statistics.mean(calls))
            pctas, pphases, _ = b.persistent_info
            mode = "lockstep" if b.lockstep_runs > 0 else "one grid per stream"
        best = min(loops, key=lambda k: loops[k][0])
        batch_s = loops[best][0]
        if best and pctas > 0:
            mode += ", one cooperative launch per CG iteration"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for gg, zz, dd in zip(grids, zs, dcs):
            gg.gradient(zz, dd)
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t0
        out["batch_64_uneven"] = {
            "grad_evals_per_s": 64 / batch_s, "timing": "median of 10 calls (wall clock)",
            "mean_grad_evals_per_s": 64 / loops[best][2],
            "sequential_grad_evals_per_s": 64 / seq_s,
            "workers": 8, "mode": mode, "elements": sum(q.n_el for q in ps),
            "cg_iters_mean": statistics.mean(i.iters for i in infos),
            "tiles": {"rows": tiles[0], "waves": tiles[1],
                      "chosen_by": "tomo_batch_autotune_tiles on other fields, untimed",
                      "candidates_ms": {"%dx%d" % (r["rows"], r["waves"]): r["ms"]
                                        for r in tile_rows}},
            "launched_iteration": {"grad_evals_per_s": 64 / loops[False][0],
                                   "cg_loop_ms": loops[False][1]},
            "persistent_iteration": {"grad_evals_per_s": 64 / loops[True][0],
                                     "cg_loop_ms": loops[True][1], "ctas": pctas,
                                     "phases": pphases, "tiles": "8x%d" % tiles[1]}}
    finally:
        for gg in grids:
            gg.close()
    return out


def run_ours(args):
    import torch

    from paper_2104_12282_gb300 import problems as P
    from paper_2104_12282_gb300 import tomo

    world, rank, local = dist_env()
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    dist = init_ranks("nccl")

    def barrier():
        if dist is not None:
            dist.barrier(device_ids=[dev.index])
        torch.cuda.synchronize()

    def slowest(x):
        return max_over_ranks(dist, x, dev)

    p = P.mbb_192x96x76(args.seed)
    fields = [P.bumpy_field(p.dims, args.seed + k) for k in range(2)]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(prec, rtol):
        return tomo.Grid.from_problem(p, precision=prec, rtol=rtol, maxit=5000,
                                      stream=stream.cuda_stream)

    # ---------------- mixed path: timed steps ----------------
    g = make(tomo.FP32, 1e-6)
    zs = [torch.tensor(f, dtype=torch.float32, device=dev) for f in fields]
    # the smoother (Chebyshev degrees, interval and cycle) chosen by the library's autotuner
    # on three other fields of the same recipe (seeds 2-4), before and outside the timed
    # region
    ztune = [torch.tensor(P.bumpy_field(p.dims, args.seed + 2 + k), dtype=torch.float32,
                          device=dev) for k in range(3)]
    tuned, _ = g.autotune(ztune, reps=2)
    del ztune
    dc = torch.empty_like(zs[0])
    dv = torch.empty_like(zs[0])
    zn = torch.empty_like(zs[0])

    def step(grid, z, dc_, dv_, zn_):
        c, info = grid.gradient(z, dc_, dv_)
        grid.oc_step(z, dc_, dv_, p.volfrac, p.move, zn_)
        return c, info

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    iters, comps = [], []
    with ClockSampler(dev.index) as clk:
        for w in range(args.warmup):
            step(g, zs[w % 2], dc, dv, zn)
        barrier()
        l0 = g.launch_count()
        clk.mark()
        for s in range(args.steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            c, info = step(g, zs[s % 2], dc, dv, zn)
            ev[s][1].record(stream)
            iters.append(info.iters)
            comps.append(c)
        barrier()
    launches = g.launch_count() - l0
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = slowest(sum(ms))
    value = whole_job_rate(world, args.steps, total_ms)
    fallbacks = g.smoother_bound()[2]

    # the same steps with the default smoother (degrees 2, 2 on the element bound)
    g.set_smoother(2, 2, 20.0)
    g.set_smoother_bound(0.0)
    g.set_cycle(0)
    for w in range(2):
        step(g, zs[w % 2], dc, dv, zn)
    ev_def = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    it_def = []
    barrier()
    for s in range(args.steps):
        flush.fill_(float(s))
        ev_def[s][0].record(stream)
        _, info_d = step(g, zs[s % 2], dc, dv, zn)
        ev_def[s][1].record(stream)
        it_def.append(info_d.iters)
    barrier()
    ms_def = [a.elapsed_time(b) for a, b in ev_def]
    value_def = whole_job_rate(world, args.steps, slowest(sum(ms_def)))
    g.set_smoother(tuned[0], tuned[1], tuned[4])
    g.set_smoother_bound(tuned[2])
    g.set_cycle(tuned[3])

    # ---------------- roofline of the smoother/product kernel ----------------
    g.profile_enable(True)
    for s in range(2):
        flush.fill_(float(s))
        step(g, zs[s % 2], dc, dv, zn)
    n_l, k_ms, k_bytes = g.profile_read()
    g.profile_enable(False)
    achieved = k_bytes / (k_ms * 1e-3) / 1e9 if k_ms > 0 else 0.0
    peak, peak_kind = peak_hbm()
    traffic = march_traffic()

    # ---------------- accuracy against the FP64 oracle (untimed) ----------------
    # the oracle's 1e-12 solve of the seed-0 field, stored by a script that calls only the
    # oracle; the mixed path's compliance and dc/dz (guarded by 1e-3 max|dc/dz|) against it
    vs_oracle = None
    gold = oracle_golden() if args.seed == 0 else None
    if gold is not None:
        scal, idx, val = gold
        c0, _ = g.gradient(zs[0], dc, dv)
        got = dc.double().cpu()[torch.tensor(idx)]
        ref = torch.tensor(val, dtype=torch.float64)
        den = torch.clamp(ref.abs(), min=1e-3 * scal["max_abs_dcdz"])
        vs_oracle = {"compliance_rel_err": abs(c0 / scal["compliance"] - 1.0),
                     "dcdz_guarded_max_rel_err": float(((got - ref).abs() / den).max()),
                     "dcdz_elements": len(idx),
                     "oracle": "FP64 Jacobi-PCG to 1e-12 on the seed-0 field "
                               "(tests/golden/fullsize_mbb_192x96x76_seed0.txt)"}

    # ---------------- e2e: host buffers through the C ABI ----------------
    zh = [torch.tensor(f, dtype=torch.float32).pin_memory() for f in fields]
    dch = torch.empty(p.n_el, dtype=torch.float32).pin_memory()
    dvh = torch.empty(p.n_el, dtype=torch.float32).pin_memory()
    znh = torch.empty(p.n_el, dtype=torch.float32).pin_memory()
    for w in range(2):
        step(g, zh[w % 2], dch, dvh, znh)
    barrier()
    e2e_ms = []
    for s in range(args.steps):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(g, zh[s % 2], dch, dvh, znh)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = slowest(sum(e2e_ms))
    e2e_value = whole_job_rate(world, args.steps, e2e_total)
    nb = 4 * p.n_el
    h2d = 4 * nb   # z (gradient), z, dcdz, dvdz (OC step)
    d2h = 3 * nb   # dcdz, dvdz (gradient), z_new (OC step)
    g.close()

    # ---------------- all-FP64 GPU path, same algorithm ----------------
    g64 = make(tomo.FP64, 1e-6)
    z64 = [torch.tensor(f, dtype=torch.float64, device=dev) for f in fields]
    dc64 = torch.empty_like(z64[0])
    dv64 = torch.empty_like(z64[0])
    zn64 = torch.empty_like(z64[0])
    step(g64, z64[0], dc64, dv64, zn64)
    ms64, c64s = [], []
    barrier()
    for s in range(args.fp64_steps):
        flush.fill_(float(s))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c, _ = step(g64, z64[s % 2], dc64, dv64, zn64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64.append(e0.elapsed_time(e1))
        c64s.append(c)
    g64.close()
    value64 = whole_job_rate(world, args.fp64_steps, slowest(sum(ms64)))
    # FP64 reference compliance at 1e-10 (untimed) for the accuracy column
    gref = make(tomo.FP64, 1e-10)
    cref = []
    for k in range(2):
        c, _ = gref.gradient(z64[k], dc64)
        cref.append(c)
    gref.close()
    cerr = max(abs(comps[s] / cref[s % 2] - 1.0) for s in range(args.steps))
    cerr64 = max(abs(c64s[s] / cref[s % 2] - 1.0) for s in range(args.fp64_steps))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    srt = sorted(ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(ms), "p50_ms": statistics.median(ms),
        "p99_ms": srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "seeds": [args.seed, args.seed + 1],
                   "step": "tomo_gradient (filter, GMG-PCG to 1e-6 from zero, sensitivity, "
                           "filter adjoints) + tomo_oc_step",
                   "precision": "FP32 products/smoothing, float-pair iterate, FP64 dots",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}", "cg_iters": iters[0],
                   "smoother": {"fine_degree": tuned[0], "coarse_degree": tuned[1],
                                "bound": tuned[2], "w_cycle_levels": tuned[3],
                                "interval_ratio": tuned[4],
                                "bound_fallbacks": fallbacks,
                                "chosen_by": "tomo_autotune_smoother_multi on the seed 2-4 "
                                             "fields of the same recipe, untimed"}},
        "default_smoother": {"value": value_def, "unit": UNIT,
                             "ms_per_step": statistics.mean(ms_def), "cg_iters": it_def[0],
                             "setting": "degrees 2, 2 on the element bound"},
        "compliance_rel_err_vs_fp64": cerr,
        "vs_fp64_oracle": vs_oracle,
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": statistics.mean(ms64),
                 "steps": args.fp64_steps, "compliance_rel_err": cerr64,
                 "note": "same algorithm in FP64 (products, smoothing, vectors), rtol 1e-6"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_march2 (fine-level FP32 product / Chebyshev smoother / residual)",
                     "launches": n_l, "avg_us": k_ms / max(1, n_l) * 1e3,
                     "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)" if peak_kind ==
                     "measured" else "fallback 6.8 TB/s"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(e2e_ms)},
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if world == 1:
        out["cpu_baseline"] = cpu_baseline(args.seed)
        out["cpu_baseline_one_core"] = cpu_baseline_one_core(args.seed)
        out.update(extras(args, dev, stream))
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
