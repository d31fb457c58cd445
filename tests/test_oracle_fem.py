"""Pins of the oracle's element stiffness and operator (no GPU).

K0 is checked against facts that do not come from the oracle itself: exact symbolic
integration of the continuum bilinear form (index notation, no Voigt matrices), the six
rigid-body modes, closed-form strain energies of uniform strains, and the cube-symmetry
block structure.  Assembly is checked against a brute-force loop and the matrix-free
product.
"""
import itertools

import numpy as np
import pytest

from oracle import fem

NU = 0.3


@pytest.fixture(scope="module")
def K0():
    return fem.unit_element_stiffness(NU)


def test_symmetric_psd_rank18(K0):
    assert np.abs(K0 - K0.T).max() <= 1e-16
    w = np.linalg.eigvalsh(K0)
    assert np.sum(np.abs(w) < 1e-12) == 6
    assert w.min() > -1e-14
    assert np.sum(w > 1e-8) == 18


def _node_xyz():
    return fem.LOCAL_NODES.astype(float)   # unit cube corners, local order x fastest


def test_rigid_body_modes_in_null_space(K0):
    X = _node_xyz()
    modes = []
    for c in range(3):                      # translations
        u = np.zeros((8, 3))
        u[:, c] = 1.0
        modes.append(u.ravel())
    for axis in np.eye(3):                  # infinitesimal rotations u = w x (x - x0)
        u = np.cross(axis, X - 0.5)
        modes.append(u.ravel())
    for m in modes:
        assert np.abs(K0 @ m).max() <= 1e-14


def test_uniform_strain_energy_closed_form(K0):
    """u = eps x on the unit cube: u^T K0 u = lam tr(eps)^2 + 2 mu eps:eps (volume 1)."""
    E = 1.0
    lam = E * NU / ((1 + NU) * (1 - 2 * NU))
    mu = E / (2 * (1 + NU))
    X = _node_xyz()
    rng = np.random.default_rng(0)
    cases = []
    for a, b in itertools.combinations_with_replacement(range(3), 2):
        eps = np.zeros((3, 3))
        eps[a, b] = eps[b, a] = 1.0
        cases.append(eps)
    S = rng.standard_normal((3, 3))
    cases.append(0.5 * (S + S.T))
    for eps in cases:
        A = eps + np.array([[0, 0.3, -0.2], [-0.3, 0, 0.1], [0.2, -0.1, 0]])  # + rotation
        u = (X @ A.T).ravel()
        exact = lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)
        assert abs(u @ K0 @ u - exact) <= 1e-13 * max(1.0, exact)


def test_matches_exact_symbolic_integration(K0):
    """Exact integration of a(u, v) = int lam div u div v + 2 mu eps(u):eps(v) over the unit
    cube with trilinear N_a, written in index notation (independent of B and D)."""
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x0:3")
    nu = sympy.Rational(3, 10)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    N = []
    for a in range(8):
        bits = [(a >> i) & 1 for i in range(3)]
        N.append(sympy.prod([x[i] if bits[i] else 1 - x[i] for i in range(3)]))
    dN = [[sympy.Poly(sympy.diff(N[a], x[i]), *x) for i in range(3)] for a in range(8)]

    def integ(poly):
        r = poly.integrate(x[0])
        r = (r.subs(x[0], 1) - r.subs(x[0], 0)) if r.free_symbols & {x[0]} else r
        expr = sympy.integrate(r.as_expr(), (x[1], 0, 1), (x[2], 0, 1))
        return expr

    G = {}
    for a in range(8):
        for b in range(8):
            for i in range(3):
                for j in range(3):
                    G[a, b, i, j] = integ(dN[a][i] * dN[b][j])
    Kex = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            lap = sum(G[a, b, k, k] for k in range(3))
            for c in range(3):
                for d in range(3):
                    v = lam * G[a, b, c, d] + mu * G[a, b, d, c] + (mu * lap if c == d else 0)
                    Kex[3 * a + c, 3 * b + d] = float(v)
    assert np.abs(K0 - Kex).max() <= 1e-14


def test_cube_symmetry_block_structure(K0):
    """In the per-component Walsh-Hadamard basis chi_m(s) = (-1)^(m.s), K0 is block
    diagonal: mode (c, m) couples only to modes (c', m') with m ^ e_c == m' ^ e_c'."""
    L = fem.LOCAL_NODES
    H = np.array([[(-1) ** int(np.dot(m, s)) for s in L] for m in L], float)
    T = np.zeros((24, 24))
    for c in range(3):
        for m in range(8):
            for s in range(8):
                T[3 * m + c, 3 * s + c] = H[m, s]
    B = T @ K0 @ T.T / 64.0
    for i in range(24):
        for j in range(24):
            mi, ci = divmod(i, 3)
            mj, cj = divmod(j, 3)
            if (mi ^ (1 << ci)) != (mj ^ (1 << cj)):
                assert abs(B[i, j]) <= 1e-15
    assert np.sum(np.abs(B) > 1e-12) == 45
    assert len(np.unique(np.round(np.abs(K0), 12))) == 10
    assert np.allclose(np.diag(K0), np.diag(K0)[0])


def test_assembly_matches_brute_force_loop(K0):
    nx, ny, nz = 3, 2, 2
    rng = np.random.default_rng(1)
    Ee = rng.uniform(0.1, 1.0, nx * ny * nz)
    h = 0.7
    K = fem.assemble(nx, ny, nz, Ee, h, K0).toarray()
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    Kb = np.zeros((3 * nn, 3 * nn))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                dofs = []
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    n = (i + ax) + (nx + 1) * ((j + ay) + (ny + 1) * (k + az))
                    for c in range(3):
                        dofs.append(c * nn + n)
                for p in range(24):
                    for q in range(24):
                        Kb[dofs[p], dofs[q]] += h * Ee[e] * K0[p, q]
    assert np.abs(K - Kb).max() <= 1e-15
    x = rng.standard_normal(3 * nn)
    y = fem.apply_elementwise(nx, ny, nz, Ee, h, K0, x)
    assert np.abs(y - Kb @ x).max() <= 1e-13
    dg = fem.diagonal_elementwise(nx, ny, nz, Ee, h, K0)
    assert np.abs(dg - np.diag(Kb)).max() <= 1e-15


def test_element_stiffness_scales_with_edge_length(K0):
    """Physical element of edge h: K_e = h E K0 (B ~ 1/h, volume ~ h^3)."""
    h = 2.5
    u = np.random.default_rng(2).standard_normal(24)
    K = fem.assemble(1, 1, 1, np.array([1.0]), h, K0).toarray()
    edof = fem.element_dofs(1, 1, 1)[0]
    Ke = K[np.ix_(edof, edof)]
    # energy of a uniform strain on a cube of edge h: (lam tr^2 + 2 mu eps:eps) h^3
    X = fem.LOCAL_NODES.astype(float) * h
    eps = np.diag([1.0, 0.0, 0.0])
    ue = (X @ eps.T).ravel()
    lam = NU / ((1 + NU) * (1 - 2 * NU))
    assert np.isclose(ue @ Ke @ ue, (lam + 2 / (2 * (1 + NU))) * h ** 3, rtol=1e-13)
    assert np.allclose(Ke, h * K0, rtol=0, atol=1e-15)
