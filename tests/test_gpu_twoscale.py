"""Two-scale coarse-graining on the GPU (tomo_coarse_grain) and the coarse state solved
with the same library, against the oracle (§III-C, Algorithm 1)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import twoscale  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a, dt):
    return torch.tensor(np.asarray(a), dtype=dt, device=DEV)


@pytest.mark.parametrize("prec", [tomo.FP32, tomo.FP64])
@pytest.mark.parametrize("dims,nb", [((20, 10, 10), 5), ((33, 17, 9), 4), ((7, 5, 3), 2),
                                     ((6, 4, 4), 1), ((5, 3, 2), 8)])
def test_coarse_grain_matches_oracle(prec, dims, nb):
    p = P.cantilever(*dims)
    z = P.random_field(p.dims, 11, 0.0, 1.0).astype(np.float32).astype(np.float64)
    ref = twoscale.coarse_grain(*dims, nb, z)
    dt = torch.float32 if prec == tomo.FP32 else torch.float64
    with tomo.Grid.from_problem(p, precision=prec) as g:
        out = torch.empty(int(np.prod(tomo.coarse_dims(*dims, nb))), dtype=dt, device=DEV)
        g.coarse_grain(_t(z, dt), nb, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
    if prec == tomo.FP64:
        assert np.abs(got - ref).max() <= 1e-15
    else:   # sums in double, one rounding to float
        assert np.array_equal(got, ref.astype(np.float32).astype(np.float64))
    if nb == 1:
        assert np.array_equal(got, z)


def test_coarse_grain_host_buffers_and_bad_block():
    p = P.cantilever(10, 5, 5)
    z = P.random_field(p.dims, 2).astype(np.float32)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        out = np.zeros(2 * 1 * 1, np.float32)
        g.coarse_grain(z, 5, out)
        assert np.array_equal(out, twoscale.coarse_grain(10, 5, 5, 5, z.astype(np.float64))
                              .astype(np.float32))
        with pytest.raises(tomo.TomoError):
            g.coarse_grain(z, 0, out)


@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
def test_coarse_state_matches_oracle(prec):
    """Algorithm 1's coarse solve: z_C from the fine grid, K_C(z_C) u_C = f_C on the coarse
    grid (element edge N_B h, rho = z_C, no filter) with tomo_solve."""
    p = P.cantilever(40, 20, 20)
    nb = 4
    z = P.bumpy_field(p.dims, 5).astype(np.float32).astype(np.float64)
    q = P.coarse_problem(p, nb)
    zc_ref = twoscale.coarse_grain(40, 20, 20, nb, z)
    dt = torch.float32 if prec == tomo.FP32 else torch.float64
    with tomo.Grid.from_problem(p, precision=prec) as g:
        zc = torch.empty(q.n_el, dtype=dt, device=DEV)
        g.coarse_grain(_t(z, dt), nb, zc)
    uc_ref, cc_ref = twoscale.coarse_state(q, zc.cpu().numpy().astype(np.float64), "direct")
    rtol = 1e-12 if prec == tomo.FP64 else 1e-6
    with tomo.Grid.from_problem(q, precision=prec, rtol=rtol, maxit=5000) as gc:
        u = torch.zeros(q.dims.n_dof, dtype=dt, device=DEV)
        info = gc.solve(zc, u)
        torch.cuda.synchronize()
    assert info.status == 0
    uc = u.cpu().numpy().astype(np.float64)
    cc = float(q.f @ uc)
    if prec == tomo.FP64:
        assert np.abs(zc.cpu().numpy() - zc_ref).max() <= 1e-15
        assert np.abs(uc - uc_ref).max() <= 1e-9 * np.abs(uc_ref).max()
        assert abs(cc / cc_ref - 1.0) <= 1e-10
    else:
        assert abs(cc / cc_ref - 1.0) <= 1e-5


def test_table1_mesh3_coarse_grid():
    """Table 1, Mesh 3 (180x90x90, N_B = 5): coarse grid 36x18x18 (dim K_C = 40,071); sampled
    block means against the oracle's definition on the full-size field."""
    p = P.cantilever(180, 90, 90)
    nb = 5
    z = P.bumpy_field(p.dims, 9).astype(np.float32)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        zc = torch.empty(36 * 18 * 18, dtype=torch.float32, device=DEV)
        g.coarse_grain(_t(z, torch.float32), nb, zc)
        torch.cuda.synchronize()
    got = zc.cpu().numpy()
    Z = z.astype(np.float64).reshape(90, 90, 180)
    rng = np.random.default_rng(0)
    for b in rng.integers(0, got.size, 64):
        I, J, K = b % 36, (b // 36) % 18, b // (36 * 18)
        ref = Z[5 * K:5 * K + 5, 5 * J:5 * J + 5, 5 * I:5 * I + 5].mean()
        assert got[b] == np.float32(ref)
    assert P.coarse_problem(p, nb).dims.n_dof == 40071


def test_warm_started_gradient_is_the_same_solve():
    """tomo_set_warm_start: along an optimisation run the next solve starts from the last
    displacement; compliance and gradient agree with a cold solve, in fewer iterations."""
    p = P.cantilever(48, 24, 24)
    z0 = P.random_field(p.dims, 13, 0.2, 1.0).astype(np.float32)
    z1 = np.clip(z0 + 0.02 * P.random_field(p.dims, 14, -1.0, 1.0), 0.0, 1.0).astype(np.float32)
    res = {}
    for warm in (False, True):
        with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
            g.set_warm_start(warm)
            dc = torch.empty(p.n_el, dtype=torch.float32, device=DEV)
            g.gradient(_t(z0, torch.float32), dc)
            c, info = g.gradient(_t(z1, torch.float32), dc)
            torch.cuda.synchronize()
            res[warm] = (c, info.iters, dc.cpu().numpy().astype(np.float64))
    (c0, it0, d0), (c1, it1, d1) = res[False], res[True]
    assert abs(c1 / c0 - 1.0) <= 2e-6
    assert np.abs(d1 - d0).max() <= 1e-4 * np.abs(d0).max()
    assert it1 < it0, (it1, it0)


def test_optimisation_driver_follows_the_oracle():
    """paper_2104_12282_gb300.optimize.run (exact gradient every iteration, warm-started
    solves, two-scale coarse step) reproduces the oracle's compliance history."""
    from oracle import topopt
    from paper_2104_12282_gb300 import optimize

    p = P.cantilever(24, 12, 12, volfrac=0.3, rmin=1.5)
    _, hist_ref = topopt.Model(p).run(6, method="direct")
    _, hist = optimize.run(p, 6, block=4, precision=tomo.FP64, rtol=1e-11)
    for r, ref in zip(hist, hist_ref):
        assert abs(r["c"] / ref["c"] - 1.0) <= 1e-8, (r, ref)
        assert r["coarse_cg_iters"] is not None and r["coarse_cg_iters"] > 0
    _, hist32 = optimize.run(p, 6, block=4, precision=tomo.FP32)
    for r, ref in zip(hist32, hist_ref):
        assert abs(r["c"] / ref["c"] - 1.0) <= 1e-5, (r, ref)


def test_synthetic_gradients_follow_the_exact_optimiser():
    """Algorithm 1 (ONSG) on Table 1's Mesh 1 (70x35x35 cantilever, block 5, 200
    iterations, N_I = N_F = 10): exact gradients on iterations 0-9 and every 10th after,
    synthetic ones (model trained online) in between.  Table 2 puts the paper's final
    compliance within 0.5 % of its standard optimiser on the cantilever meshes; this reading
    of the model's inputs (features documented in onsg.py) is held to 3 % of the exact
    optimiser run with the same library (measured -1.3 %)."""
    from paper_2104_12282_gb300 import onsg
    from paper_2104_12282_gb300.optimize import paper_cantilever

    p = paper_cantilever(1)
    _, h_ex, c_ex = onsg.run(p, 200, block=5, exact_only=True)
    _, h_sg, c_sg = onsg.run(p, 200, block=5)
    assert sum(r["exact"] for r in h_ex) == 200
    assert sum(r["exact"] for r in h_sg) == 10 + 19
    assert all(r["c"] is not None for r in h_sg if r["exact"])
    assert np.isfinite(c_sg) and abs(c_sg / c_ex - 1.0) <= 0.03, (c_sg, c_ex)
