"""Writes the full-size oracle goldens: the FP64 oracle's exact gradient on the two large
workloads, where the oracle solves too slowly to run inside a test.

    python tests/golden/make_fullsize_goldens.py mbb      # 192x96x76, bumpy field seed 0
    python tests/golden/make_fullsize_goldens.py cant     # 96x48x48 cantilever, uniform start

Only ``oracle/`` computes: the state K_ff u_f = f_f (Eq. 4) by its Jacobi-PCG to a relative
residual of 1e-12 (the true residual f - K u is recomputed with the oracle's operator and
stored), the compliance c = f^T u (Eq. 4) and the filtered sensitivity dc/dz = P^T dc/drho
(Eq. 5 with the SIMP chain rule).  ``problems`` supplies the seeded inputs (supports, load,
design field); the design is rounded to float32 first, as the GPU tests pass it.  Each
golden file stores c and dc/dz at 1,024 elements drawn by numpy default_rng(12282) plus the
element of largest |dc/dz|, with max |dc/dz| for the guarded relative error.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fem, solve, topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

CASES = {
    "mbb": ("fullsize_mbb_192x96x76_seed0.txt", lambda: P.mbb_192x96x76(0),
            "192x96x76 MBB-type block, bumpy field seed 0 (volfrac 0.12, rmin 2.5)"),
    "cant": ("fullsize_cantilever_96x48x48_uniform.txt", P.cantilever_96x48x48,
             "96x48x48 cantilever, uniform start z = 0.3 (rmin 1.5)"),
}
N_SAMPLE = 1024


def run(case: str) -> str:
    fname, make, what = CASES[case]
    p = make()
    d = p.dims
    m = topopt.Model(p)
    z = np.asarray(p.z0, np.float64).astype(np.float32).astype(np.float64)
    t0 = time.time()
    rho = m.filter(z)
    E = m.modulus(rho)
    diag = fem.diagonal_elementwise(d.nx, d.ny, d.nz, E, p.h, m.K0, m.edof)
    count = [0]

    def apply_full(v):
        count[0] += 1
        if count[0] % 500 == 0:
            print(f"  {case}: {count[0]} products, {time.time() - t0:.0f} s", flush=True)
        return fem.apply_elementwise(d.nx, d.ny, d.nz, E, p.h, m.K0, v, m.edof)

    u, iters, rel = solve.solve_pcg_matfree(apply_full, diag, p.f, m.fixed, 1e-12, 400000)
    true_rel = float(np.linalg.norm(p.f - m.apply(E, u)) / np.linalg.norm(p.f))
    c = float(p.f @ u)
    dcdz = m.filter_T(m.sensitivity(rho, u))
    rng = np.random.default_rng(12282)
    idx = np.unique(np.concatenate([rng.choice(d.n_el, N_SAMPLE, replace=False),
                                    [int(np.argmax(np.abs(dcdz)))]]))
    secs = time.time() - t0
    path = os.path.join(HERE, fname)
    with open(path, "w") as fh:
        fh.write(f"# FP64 oracle exact gradient: {what}\n")
        fh.write(f"# written by: python tests/golden/make_fullsize_goldens.py {case}\n")
        fh.write("# state: oracle Jacobi-PCG (solve.solve_pcg_matfree) to 1e-12; compliance\n")
        fh.write("# c = f^T u (Eq. 4); dcdz = P^T dc/drho (Eq. 5, SIMP chain rule); design z\n")
        fh.write("# rounded to float32 before the oracle runs\n")
        fh.write(f"# oracle time {secs:.0f} s on {os.cpu_count()} host cores\n")
        fh.write(f"n_el {d.n_el}\n")
        fh.write(f"n_dof {d.n_dof}\n")
        fh.write(f"compliance {c!r}\n")
        fh.write(f"pcg_iterations {iters}\n")
        fh.write(f"pcg_rel_res {float(rel)!r}\n")
        fh.write(f"true_rel_res {true_rel!r}\n")
        fh.write(f"max_abs_dcdz {float(np.abs(dcdz).max())!r}\n")
        fh.write("# element dcdz\n")
        for e in idx:
            fh.write(f"{int(e)} {float(dcdz[e])!r}\n")
    print(f"{case}: c = {c!r}, {iters} iterations, true rel. residual {true_rel:.2e}, "
          f"{secs:.0f} s -> {path}", flush=True)
    return path


if __name__ == "__main__":
    for c in sys.argv[1:] or list(CASES):
        run(c)
