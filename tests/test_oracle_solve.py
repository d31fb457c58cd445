"""Pins of the oracle's state solve (no GPU): patch test, energy identity, direct vs PCG,
matrix-free vs assembled operator, slender-cantilever deflection against beam theory."""
import numpy as np
import pytest

from oracle import fem, solve
from paper_2104_12282_gb300 import problems as P

NU = 0.3


@pytest.fixture(scope="module")
def K0():
    return fem.unit_element_stiffness(NU)


def test_patch_test_linear_field(K0):
    """Uniform material, u = A x + b prescribed on the boundary: the interior reproduces the
    linear field and u^T K u equals the closed-form strain energy times the volume."""
    nx, ny, nz, h = 4, 3, 3, 0.5
    d = P.GridDims(nx, ny, nz)
    nn = d.n_nodes
    K = fem.assemble(nx, ny, nz, np.ones(d.n_el), h, K0)
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], 1) * h
    A = np.array([[0.01, 0.02, -0.03], [0.005, -0.02, 0.01], [0.015, 0.0, 0.025]])
    b = np.array([0.1, -0.2, 0.3])
    U = X @ A.T + b
    uex = np.concatenate([U[:, c] for c in range(3)])
    ib, jb, kb = i.ravel(), j.ravel(), k.ravel()
    bnd = (ib == 0) | (ib == nx) | (jb == 0) | (jb == ny) | (kb == 0) | (kb == nz)
    fixed = np.tile(bnd, 3)
    ub = np.where(fixed, uex, 0.0)
    uI = solve.solve_direct(K, -(K @ ub), fixed)
    u = uI + ub
    assert np.abs(u - uex).max() <= 1e-12
    eps = 0.5 * (A + A.T)
    lam = NU / ((1 + NU) * (1 - 2 * NU))
    mu = 1 / (2 * (1 + NU))
    energy = (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)) * (nx * ny * nz * h ** 3)
    assert np.isclose(u @ (K @ u), energy, rtol=1e-12)


def test_energy_identity_and_solvers_agree(K0):
    p = P.cantilever(8, 4, 4)
    d = p.dims
    rng = np.random.default_rng(3)
    E = rng.uniform(0.05, 1.0, d.n_el)
    K = fem.assemble(d.nx, d.ny, d.nz, E, p.h, K0)
    u = solve.solve_direct(K, p.f, p.fixed)
    c = p.f @ u
    assert np.isclose(c, u @ (K @ u), rtol=1e-12)
    free = p.fixed == 0
    assert np.abs((K @ u - p.f)[free]).max() <= 1e-12 * np.abs(p.f).max() * 1e3
    assert np.all(u[p.fixed == 1] == 0.0)
    u2, it, rel = solve.solve_pcg_csr(K, p.f, p.fixed, tol=1e-12)
    assert rel <= 1e-12 and it > 10
    assert np.abs(u2 - u).max() <= 1e-9 * np.abs(u).max()
    diag = fem.diagonal_elementwise(d.nx, d.ny, d.nz, E, p.h, K0)
    u3, it3, rel3 = solve.solve_pcg_matfree(
        lambda v: fem.apply_elementwise(d.nx, d.ny, d.nz, E, p.h, K0, v), diag, p.f, p.fixed)
    assert rel3 <= 1e-12
    assert np.abs(u3 - u).max() <= 1e-9 * np.abs(u).max()


@pytest.mark.slow
def test_slender_cantilever_against_timoshenko(K0):
    """L/H = 16 cantilever, tip traction on the end face: the hex8 tip deflection converges
    to Timoshenko beam theory PL^3/(3EI) + PL/(kGA), k = 5/6, from below (hex8 is stiff in
    bending), with the error shrinking under refinement and below 2% at 8 elements deep."""
    errs = []
    for n in (2, 4, 8):
        nx, ny, nz = 16 * n, n, n
        p = P.cantilever(nx, ny, nz)
        d = p.dims
        nn = d.n_nodes
        f = np.zeros(d.n_dof)
        wy = P._edge_weights(ny) / ny
        wz = P._edge_weights(nz) / nz
        for kk in range(nz + 1):
            for jj in range(ny + 1):
                f[2 * nn + d.node(nx, jj, kk)] = -wy[jj] * wz[kk]
        K = fem.assemble(nx, ny, nz, np.ones(d.n_el), 1.0, K0)
        u = solve.solve_direct(K, f, p.fixed)
        tip = sum(-u[2 * nn + d.node(nx, jj, kk)] * wy[jj] * wz[kk]
                  for kk in range(nz + 1) for jj in range(ny + 1))
        L, H, W = nx, nz, ny
        G = 1 / (2 * (1 + NU))
        I = W * H ** 3 / 12
        theory = L ** 3 / (3 * I) + L / (5 / 6 * G * W * H)
        errs.append(tip / theory - 1.0)
    assert errs[0] < errs[1] < errs[2] < 0.0
    assert abs(errs[2]) < 0.02
