"""Pins of the oracle's sensitivities and loop (no GPU): central finite differences of the
compliance with respect to rho and to z (through the filter), and loop invariants."""
import numpy as np
import pytest

from oracle import topopt
from paper_2104_12282_gb300 import problems as P


def _compliance_of_rho(m, rho):
    u, _, _ = m.solve(m.modulus(rho), "direct")
    return m.p.f @ u, u


@pytest.mark.parametrize("dims", [(3, 2, 2), (4, 2, 2)])
def test_sensitivity_matches_central_differences(dims):
    p = P.cantilever(*dims, rmin=1.0, h=0.8)
    m = topopt.Model(p)
    rho = np.random.default_rng(4).uniform(0.3, 1.0, p.n_el)
    c, u = _compliance_of_rho(m, rho)
    dc = m.sensitivity(rho, u)
    for e in range(p.n_el):
        step = 1e-6 * rho[e]
        rp = rho.copy()
        rm = rho.copy()
        rp[e] += step
        rm[e] -= step
        fd = (_compliance_of_rho(m, rp)[0] - _compliance_of_rho(m, rm)[0]) / (2 * step)
        assert abs(fd - dc[e]) <= 1e-6 * abs(dc[e]), (e, fd, dc[e])
    assert np.all(dc < 0)


def test_filtered_gradient_matches_central_differences():
    """dc/dz = P^T dc/drho with a non-trivial filter (rmin 1.5, boundary-truncated rows)."""
    p = P.cantilever(4, 3, 2, rmin=1.5)
    m = topopt.Model(p)
    z = np.random.default_rng(5).uniform(0.3, 1.0, p.n_el)
    g = m.gradient(z, "direct")

    def cz(zz):
        return _compliance_of_rho(m, m.filter(zz))[0]

    for e in range(0, p.n_el, 3):
        step = 1e-6 * z[e]
        zp = z.copy()
        zm = z.copy()
        zp[e] += step
        zm[e] -= step
        fd = (cz(zp) - cz(zm)) / (2 * step)
        assert abs(fd - g["dcdz"][e]) <= 1e-6 * abs(g["dcdz"][e])
    # wrong-adjoint guard: the forward filter applied to dc/drho gives a different vector
    assert np.abs(m.filter(g["dc_drho"]) - g["dcdz"]).max() > 1e-6 * np.abs(g["dcdz"]).max()


def test_gradient_direct_and_pcg_agree():
    p = P.cantilever(10, 5, 5, rmin=1.5)
    m = topopt.Model(p)
    z = P.random_field(p.dims, 6, 0.2, 1.0)
    a = m.gradient(z, "direct")
    b = m.gradient(z, "pcg", tol=1e-12)
    assert abs(a["c"] - b["c"]) <= 1e-10 * a["c"]
    assert np.abs(a["dcdz"] - b["dcdz"]).max() <= 1e-9 * np.abs(a["dcdz"]).max()


def test_oc_loop_invariants():
    """Cantilever from the uniform design: the filtered volume meets V_max once the move
    limit allows, and the compliance drops over the first iterations."""
    p = P.cantilever(12, 6, 6, volfrac=0.3, rmin=1.5)
    m = topopt.Model(p)
    z, hist = m.run(6, method="direct")
    cs = [h["c"] for h in hist]
    assert cs[-1] < cs[0]
    assert all(b <= a * (1 + 1e-9) for a, b in zip(cs[1:4], cs[2:5]))
    vmax = m.vmax()
    for h in hist:
        assert h["vol"] <= vmax * (1 + 1e-6)
    assert np.all((z >= 0) & (z <= 1))
    rho = m.filter(z)
    assert np.isclose(m.v @ rho, vmax, rtol=1e-7)
