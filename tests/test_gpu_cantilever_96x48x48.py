"""The 96x48x48 cantilever (221,184 elements, 698,691 DOFs; volfrac 0.3, rmin 1.5, uniform
start): 50 OC iterations on an FP32 grid (GMG-PCG, rtol 1e-6).

* The compliance history follows the all-FP64 GPU run of the same algorithm at rtol 1e-10
  within 1e-5 relative at every iteration (the FP64 grid is itself held to the oracle at
  1e-10 on the grids the oracle solves).
* The first gradient is held to the oracle's own 1e-12 solve of this workload (stored in
  tests/golden/; the oracle takes about a minute for it, too long for a test).
* At the first, a middle and the last iteration the oracle checks the step with its own
  FP64 operator (it cannot solve 698k DOFs in seconds): the residual of the displacement,
  compliance and energy identity, the gradient composed from the same displacement, and
  the OC update on the same inputs.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from oracle import topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402
import large_grid_checks as L  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")
CHECK_AT = (0, 24, 49)


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _trajectory(p, precision, rtol, keep=()):
    dt = torch.float64 if precision == tomo.FP64 else torch.float32
    cs, kept = [], {}
    with tomo.Grid.from_problem(p, precision=precision, rtol=rtol, maxit=5000,
                                mg_levels=p.meta["mg_levels"]) as g:
        z = torch.tensor(p.z0, dtype=dt, device=DEV)
        dc, dv, zn = torch.empty_like(z), torch.empty_like(z), torch.empty_like(z)
        u = torch.empty(p.dims.n_dof, dtype=dt, device=DEV)
        for k in range(p.meta["oc_iters"]):
            c, info = g.gradient(z, dc, dv)
            assert info.status == 0 and info.rel_res <= rtol
            change = g.oc_step(z, dc, dv, p.volfrac, p.move, zn)
            cs.append(c)
            if k in keep:
                g.get_displacement(u)
                torch.cuda.synchronize()
                kept[k] = dict(z=H(z), u=H(u), c=c, dcdz=H(dc), dvdz=H(dv), z_new=H(zn),
                               change=change, iters=info.iters)
            z, zn = zn, z
    return np.array(cs), kept


@pytest.fixture(scope="module")
def runs():
    p = P.cantilever_96x48x48()
    assert (p.dims.n_el, p.dims.n_dof) == (221184, 698691)
    c32, kept = _trajectory(p, tomo.FP32, 1e-6, CHECK_AT)
    c64, _ = _trajectory(p, tomo.FP64, 1e-10)
    return p, topopt.Model(p), c32, c64, kept


def test_compliance_history_follows_the_fp64_run(runs):
    p, _, c32, c64, _ = runs
    assert len(c32) == len(c64) == 50
    rel = np.abs(c32 / c64 - 1.0)
    assert rel.max() <= 1e-5, rel.max()
    assert c32[-1] < 0.5 * c32[0]     # the optimisation made progress


def test_first_gradient_matches_the_oracle_golden(runs):
    """Iteration 0 (uniform start) against the FP64 oracle's own 1e-12 solve, stored by
    tests/golden/make_fullsize_goldens.py cant."""
    p, _, _, _, kept = runs
    L.check_golden("fullsize_cantilever_96x48x48_uniform.txt", kept[0]["c"], kept[0]["dcdz"],
                   p.dims.n_el)


@pytest.mark.parametrize("k", CHECK_AT)
def test_step_satisfies_the_oracle(runs, k):
    p, m, _, _, kept = runs
    s = kept[k]
    z = s["z"]
    L.check_solve(p, m, z, s["u"], s["c"])
    L.check_gradient(m, z, s["u"], s["dcdz"], s["dvdz"])
    L.check_oc(p, m, z, s["dcdz"], s["dvdz"], s["z_new"], s["change"])
