"""Pins of the oracle's density filter (no GPU)."""
import numpy as np
import pytest

from oracle import filt


def _brute_H(nx, ny, nz, rmin):
    n = nx * ny * nz
    H = np.zeros((n, n))
    for a in range(n):
        ia, ja, ka = a % nx, (a // nx) % ny, a // (nx * ny)
        for b in range(n):
            ib, jb, kb = b % nx, (b // nx) % ny, b // (nx * ny)
            dist = np.sqrt((ia - ib) ** 2 + (ja - jb) ** 2 + (ka - kb) ** 2)
            H[a, b] = max(0.0, rmin - dist)
    return H


@pytest.mark.parametrize("rmin", [1.5, 2.5, 1.2])
def test_matrix_matches_brute_force(rmin):
    nx, ny, nz = 5, 4, 3
    H, Hs = filt.filter_matrix(nx, ny, nz, rmin)
    Hb = _brute_H(nx, ny, nz, rmin)
    assert np.abs(H.toarray() - Hb).max() <= 1e-15
    assert np.allclose(Hs, Hb.sum(1), rtol=1e-15)


def test_interior_neighbour_counts():
    assert len(filt.stencil_offsets(1.5)) == 19
    assert len(filt.stencil_offsets(2.5)) == 81
    assert len(filt.stencil_offsets(1.0)) == 1


def test_rows_sum_to_one_and_identity_below_one():
    nx, ny, nz = 6, 5, 4
    z = np.random.default_rng(0).uniform(size=nx * ny * nz)
    assert np.allclose(filt.filter_forward(nx, ny, nz, 2.5, np.ones(nx * ny * nz)), 1.0,
                       rtol=0, atol=1e-15)
    assert np.array_equal(filt.filter_forward(nx, ny, nz, 1.0, z), z)
    assert np.abs(filt.filter_forward(nx, ny, nz, 0.7, z) - z).max() <= 2e-16


@pytest.mark.parametrize("rmin", [1.5, 2.5, 5.5, 7.2])
def test_forward_and_transpose_against_dense(rmin):
    """Includes radii whose offsets exceed the grid (7 x 4 x 3 with rmin 5.5, 7.2)."""
    nx, ny, nz = 7, 4, 3
    H, Hs = filt.filter_matrix(nx, ny, nz, rmin)
    Pd = H.toarray() / Hs[:, None]
    rng = np.random.default_rng(1)
    z = rng.uniform(size=nx * ny * nz)
    x = rng.standard_normal(nx * ny * nz)
    assert np.abs(filt.filter_forward(nx, ny, nz, rmin, z) - Pd @ z).max() <= 1e-15
    assert np.abs(filt.filter_transpose(nx, ny, nz, rmin, x) - Pd.T @ x).max() <= 1e-14
    # P is not symmetric near the boundary, so the transpose differs from the forward map
    assert np.abs(Pd - Pd.T).max() > 1e-3
    sample = np.array([0, 5, 17, 40, nx * ny * nz - 1])
    assert np.abs(filt.filter_forward_at(nx, ny, nz, rmin, z, sample) - (Pd @ z)[sample]).max() <= 1e-15


def test_volume_gradient_is_adjoint():
    """d(v^T P z)/dz = P^T v; the map is linear so a unit perturbation is exact."""
    nx, ny, nz, rmin = 6, 3, 3, 1.5
    v = np.full(nx * ny * nz, 0.125)
    w = filt.filter_transpose(nx, ny, nz, rmin, v)
    z = np.random.default_rng(2).uniform(size=v.size)
    base = v @ filt.filter_forward(nx, ny, nz, rmin, z)
    for e in (0, 7, 30, v.size - 1):
        dz = np.zeros_like(z)
        dz[e] = 1.0
        assert np.isclose(v @ filt.filter_forward(nx, ny, nz, rmin, z + dz) - base, w[e],
                          rtol=1e-12)
