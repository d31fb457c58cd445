"""Two-scale coarse-graining (§III-C, Algorithm 1): oracle pins independent of the oracle's
own code path.  z_C is a plain definition (block means), pinned by a brute-force element
loop, conservation and the uniform case; the coarse grid is pinned by Table 1's K_C
dimensions; K_C is pinned by the N_B = 1 identity the paper states (K_C = K)."""
import os

import numpy as np
import pytest

from oracle import topopt, twoscale
from paper_2104_12282_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_mesh_stats.txt")


def _brute(nx, ny, nz, nb, z):
    cx, cy, cz = -(-nx // nb), -(-ny // nb), -(-nz // nb)
    s = np.zeros(cx * cy * cz)
    n = np.zeros(cx * cy * cz)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                b = (i // nb) + cx * ((j // nb) + cy * (k // nb))
                s[b] += z[i + nx * (j + ny * k)]
                n[b] += 1
    return s / n, n


@pytest.mark.parametrize("dims,nb", [((6, 4, 2), 2), ((7, 5, 3), 2), ((10, 5, 5), 5),
                                     ((9, 4, 7), 4), ((3, 3, 3), 1), ((4, 2, 3), 8)])
def test_block_means_match_element_loop(dims, nb):
    z = np.random.default_rng(1).uniform(0, 1, size=int(np.prod(dims)))
    ref, _ = _brute(*dims, nb, z)
    assert np.allclose(twoscale.coarse_grain(*dims, nb, z), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dims,nb", [((12, 6, 6), 3), ((13, 7, 5), 4)])
def test_block_means_conserve_the_total_and_keep_uniform_fields(dims, nb):
    z = np.random.default_rng(2).uniform(0, 1, size=int(np.prod(dims)))
    zc = twoscale.coarse_grain(*dims, nb, z)
    _, counts = _brute(*dims, nb, z)
    assert abs(counts @ zc - z.sum()) <= 1e-12 * z.sum()
    assert np.allclose(twoscale.coarse_grain(*dims, nb, np.full(z.size, 0.37)), 0.37,
                       rtol=0, atol=1e-15)


def test_coarse_grids_match_table1():
    """dim K_C = 3 (nx/N_B + 1)(ny/N_B + 1)(nz/N_B + 1) as printed (3K, 8K, 40K)."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for name, nx, ny, nz, nb, _, _, kcdim in rows:
        p = P.cantilever(int(nx), int(ny), int(nz))
        q = P.coarse_problem(p, int(nb))
        assert q.dims.n_dof == {"3K": 2880, "8K": 7623, "40K": 40071}[kcdim], name
        assert q.h == p.h * int(nb)


def test_block_size_one_gives_the_fine_problem():
    """N_B = 1: z_C = z and, with P = I (rmin <= 1), K_C = K, so u_C is the fine state."""
    p = P.cantilever(8, 4, 4, rmin=1.0)
    z = P.random_field(p.dims, 3)
    assert np.array_equal(twoscale.coarse_grain(8, 4, 4, 1, z), z)
    q = P.coarse_problem(p, 1)
    assert np.array_equal(q.fixed, p.fixed) and np.array_equal(q.f, p.f)
    uc, cc = twoscale.coarse_state(q, z, "direct")
    g = topopt.Model(p).gradient(z, "direct")
    assert np.allclose(uc, g["u"], rtol=0, atol=1e-12 * np.abs(g["u"]).max())
    assert abs(cc / g["c"] - 1.0) <= 1e-12


def test_coarse_load_keeps_the_total_force():
    for p in (P.cantilever(20, 10, 10), P.mbb_block(16, 8, 6)):
        for nb in (2, 3, 5):
            q = P.coarse_problem(p, nb)
            assert abs(q.f.sum() + 1.0) <= 1e-12
            assert q.meta["fine"] == (p.dims.nx, p.dims.ny, p.dims.nz)


def test_custom_loads_are_not_coarsened_silently():
    p = P.uneven_cantilever_batch(0, 1)[0]
    with pytest.raises(ValueError):
        P.coarse_problem(p, 2)
