"""General objective through the adjoint (Eq. 3) on the GPU, against the oracle."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a, dt):
    return torch.tensor(np.asarray(a), dtype=dt, device=DEV)


@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
@pytest.mark.parametrize("kind", ["cantilever", "mbb"])
def test_adjoint_gradient_matches_oracle(prec, kind):
    p = P.cantilever(16, 8, 8, rmin=1.5) if kind == "cantilever" else P.mbb_block(17, 9, 7)
    d = p.dims
    rng = np.random.default_rng(31)
    z = P.random_field(d, 32, 0.1, 1.0).astype(np.float32).astype(np.float64)
    l = rng.standard_normal(d.n_dof).astype(np.float32).astype(np.float64)
    ref = topopt.Model(p).adjoint_gradient(z, l, "direct")
    dt = torch.float32 if prec == tomo.FP32 else torch.float64
    rtol = 1e-12 if prec == tomo.FP64 else 1e-6
    with tomo.Grid.from_problem(p, precision=prec, rtol=rtol, maxit=5000) as g:
        dj = torch.empty(d.n_el, dtype=dt, device=DEV)
        J, iu, il = g.adjoint_gradient(_t(z, dt), _t(l, dt), dj)
        u = torch.empty(d.n_dof, dtype=dt, device=DEV)
        g.get_displacement(u)
        torch.cuda.synchronize()
    assert iu.status == 0 and il.status == 0 and iu.iters > 0 and il.iters > 0
    got = dj.cpu().numpy().astype(np.float64)
    scale = np.abs(ref["dJdz"]).max()
    if prec == tomo.FP64:
        assert abs(J / ref["J"] - 1.0) <= 1e-10
        assert np.abs(got - ref["dJdz"]).max() <= 1e-9 * scale
        assert np.abs(u.cpu().numpy() - ref["u"]).max() <= 1e-9 * np.abs(ref["u"]).max()
    else:
        # J = l^T u with a signed l: measure its error against sum |l||u| (no cancellation credit)
        assert abs(J - ref["J"]) <= 1e-5 * (np.abs(l) @ np.abs(ref["u"]))
        assert np.abs(got - ref["dJdz"]).max() <= 1e-4 * scale


def test_compliance_is_the_self_adjoint_case_on_the_gpu():
    p = P.cantilever(16, 8, 8, rmin=1.5)
    z = P.random_field(p.dims, 3, 0.1, 1.0)
    with tomo.Grid.from_problem(p, precision=tomo.FP64, rtol=1e-12, maxit=5000) as g:
        dc = torch.empty(p.n_el, dtype=torch.float64, device=DEV)
        dj = torch.empty_like(dc)
        c, _ = g.gradient(_t(z, torch.float64), dc)
        J, _, _ = g.adjoint_gradient(_t(z, torch.float64), _t(p.f, torch.float64), dj)
        torch.cuda.synchronize()
    assert abs(J / c - 1.0) <= 1e-11
    d0, d1 = dc.cpu().numpy(), dj.cpu().numpy()
    assert np.abs(d1 - d0).max() <= 1e-9 * np.abs(d0).max()


def test_gradient_after_adjoint_uses_the_load_again():
    """The adjoint solve swaps the right-hand side; the next compliance gradient must see f."""
    p = P.cantilever(12, 6, 6)
    z = P.random_field(p.dims, 4, 0.1, 1.0).astype(np.float32)
    l = np.random.default_rng(5).standard_normal(p.dims.n_dof).astype(np.float32)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        dc = torch.empty(p.n_el, dtype=torch.float32, device=DEV)
        c0, _ = g.gradient(_t(z, torch.float32), dc)
        g.adjoint_gradient(_t(z, torch.float32), _t(l, torch.float32), torch.empty_like(dc))
        c1, _ = g.gradient(_t(z, torch.float32), dc)
    assert c0 == c1


def test_zero_adjoint_load_gives_zero_gradient():
    p = P.cantilever(8, 4, 4)
    z = P.random_field(p.dims, 6, 0.2, 1.0).astype(np.float32)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        dj = torch.full((p.n_el,), 7.0, dtype=torch.float32, device=DEV)
        J, iu, il = g.adjoint_gradient(_t(z, torch.float32),
                                       torch.zeros(p.dims.n_dof, dtype=torch.float32, device=DEV),
                                       dj)
        torch.cuda.synchronize()
    assert J == 0.0 and il.iters == 0 and iu.status == 0
    assert torch.count_nonzero(dj).item() == 0
