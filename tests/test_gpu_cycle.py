"""Multigrid cycle shape (tomo_set_cycle): a W-cycle at levels 1 and 2 solves the same
system to the same tolerance as the V-cycle (checked against the oracle's direct solve),
in no more CG iterations on a high-contrast design; switching back restores the V-cycle's
result bitwise; a grid with W-cycle levels runs alone in a batch (not lockstep) and gives
its result alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _contrast_field(p, seed):
    """Densities near 0 or 1 (as OC-evolved designs): the rediscretised coarse operators
    are weakest there."""
    r = np.random.default_rng(seed)
    z = np.where(r.random(p.n_el) < 0.35, 1.0, 0.02).astype(np.float32)
    return z, torch.tensor(z, device=DEV)


def _grad(g, zt):
    dc = torch.empty_like(zt)
    c, info = g.gradient(zt, dc)
    torch.cuda.synchronize()
    return c, info, dc.cpu().numpy()


def test_w_cycle_solves_to_tolerance_and_switches_back():
    p = P.cantilever(48, 24, 24)
    z, zt = _contrast_field(p, 5)
    ref = topopt.Model(p).gradient(z.astype(np.float64), "direct")
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        assert g.counts()[2] >= 5 and g.cycle() == 0
        cv, iv, dv = _grad(g, zt)
        g.set_cycle(0b110)
        assert g.cycle() == 6
        cw, iw, dw = _grad(g, zt)
        g.set_cycle(0)
        cv2, iv2, dv2 = _grad(g, zt)
    for c, info, d in ((cv, iv, dv), (cw, iw, dw)):
        assert info.status == 0 and info.rel_res <= 1e-6
        assert abs(c / ref["c"] - 1.0) <= 1e-5
        scale = np.abs(ref["dcdz"]).max()
        assert np.abs(d - ref["dcdz"]).max() <= 1e-4 * scale
    assert iw.iters <= iv.iters
    assert cv2 == cv and iv2.iters == iv.iters and np.array_equal(dv2, dv)


def test_cycle_mask_needs_a_multigrid_grid():
    p = P.cantilever(12, 6, 6)
    with tomo.Grid.from_problem(p, precision=tomo.FP32, precond=tomo.PRECOND_JACOBI) as g:
        with pytest.raises(tomo.TomoError):
            g.set_cycle(2)
        g.set_cycle(0)


def test_w_cycle_grid_runs_alone_in_a_batch():
    ps = P.uneven_cantilever_batch(7, 3)
    zs = [_contrast_field(p, 40 + i)[1] for i, p in enumerate(ps)]
    grids = [tomo.Grid.from_problem(p, precision=tomo.FP32) for p in ps]
    try:
        grids[1].set_cycle(2)
        alone = [_grad(g, z) for g, z in zip(grids, zs)]
        with tomo.Batch(workers=2) as b:
            for g in grids:
                b.append(g)
            dcs = [torch.empty_like(z) for z in zs]
            cs, infos = b.gradient(zs, dcs)
            torch.cuda.synchronize()
            assert b.lockstep_runs == 0        # one grid per stream
        for (c, info, d), c2, i2, d2 in zip(alone, cs, infos, dcs):
            assert c2 == c and i2.iters == info.iters
            assert np.array_equal(d2.cpu().numpy(), d)
    finally:
        for g in grids:
            g.close()
