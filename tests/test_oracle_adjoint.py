"""General adjoint gradient (Eq. 3) for a linear functional J = l^T u of the state: pinned
by central finite differences of J(z) and by the compliance special case (l = f)."""
import numpy as np
import pytest

from oracle import topopt
from paper_2104_12282_gb300 import problems as P


def _J(m, z, l):
    rho = m.filter(z)
    u, _, _ = m.solve(m.modulus(rho), "direct")
    return float(np.where(m.fixed, 0.0, l) @ u)


@pytest.mark.parametrize("dims,rmin", [((3, 2, 2), 1.0), ((4, 3, 2), 1.5)])
def test_adjoint_gradient_matches_central_differences(dims, rmin):
    p = P.cantilever(*dims, rmin=rmin, h=0.7)
    m = topopt.Model(p)
    rng = np.random.default_rng(8)
    z = rng.uniform(0.3, 1.0, p.n_el)
    # a non-self-adjoint functional: a signed combination of displacements away from the load
    l = rng.standard_normal(p.dims.n_dof)
    g = m.adjoint_gradient(z, l, "direct")
    assert abs(g["J"] - _J(m, z, l)) <= 1e-12 * abs(g["J"])
    for e in range(p.n_el):
        step = 1e-6 * z[e]
        zp, zm = z.copy(), z.copy()
        zp[e] += step
        zm[e] -= step
        fd = (_J(m, zp, l) - _J(m, zm, l)) / (2 * step)
        assert abs(fd - g["dJdz"][e]) <= 1e-6 * np.abs(g["dJdz"]).max(), (e, fd, g["dJdz"][e])


def test_compliance_is_the_self_adjoint_case():
    p = P.cantilever(6, 3, 3, rmin=1.5)
    m = topopt.Model(p)
    z = np.random.default_rng(9).uniform(0.2, 1.0, p.n_el)
    g = m.gradient(z, "direct")
    a = m.adjoint_gradient(z, p.f, "direct")
    assert abs(a["J"] / g["c"] - 1.0) <= 1e-13
    assert np.allclose(a["lam"], g["u"], rtol=0, atol=1e-12 * np.abs(g["u"]).max())
    assert np.allclose(a["dJdz"], g["dcdz"], rtol=0, atol=1e-12 * np.abs(g["dcdz"]).max())
