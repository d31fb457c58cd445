"""Input generators: grid conventions against Table 1, loads and supports."""
import os

import numpy as np

from paper_2104_12282_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_mesh_stats.txt")


def _parse_count(s):
    mult = {"K": 1e3, "M": 1e6}[s[-1]]
    return float(s[:-1]) * mult, s


def _rounds_to(value, printed):
    """True if `value` prints as `printed` at the paper's precision (e.g. 1.5M, 276K)."""
    target, s = _parse_count(printed)
    unit = {"K": 1e3, "M": 1e6}[s[-1]]
    decimals = len(s[:-1].split(".")[1]) if "." in s else 0
    return round(value / unit, decimals) == round(target / unit, decimals)


def test_table1_dof_counts():
    """Hex8 with 3 DOFs per node reproduces every printed count of Table 1 (cantilever):
    #DVs = nx*ny*nz, dim K = 3(nx+1)(ny+1)(nz+1), dim K_C = same on the N_B-coarsened grid."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for name, nx, ny, nz, nb, dvs, kdim, kcdim in rows:
        d = P.GridDims(int(nx), int(ny), int(nz))
        nb = int(nb)
        assert d.nx % nb == 0 and d.ny % nb == 0 and d.nz % nb == 0
        dc = P.GridDims(d.nx // nb, d.ny // nb, d.nz // nb)
        assert _rounds_to(d.n_el, dvs), (name, d.n_el, dvs)
        assert _rounds_to(d.n_dof, kdim), (name, d.n_dof, kdim)
        assert _rounds_to(dc.n_dof, kcdim), (name, dc.n_dof, kcdim)
        assert d.nx == 2 * d.ny == 2 * d.nz


def test_exact_counts_of_named_grids():
    assert P.GridDims(70, 35, 35).n_dof == 276048
    assert P.GridDims(100, 50, 50).n_dof == 788103
    assert P.GridDims(180, 90, 90).n_dof == 4496583
    d3 = P.GridDims(192, 96, 76)
    assert d3.n_el == 1400832 and d3.n_nodes == 1441517 and d3.n_dof == 4324551


def test_cantilever_supports_and_load():
    p = P.cantilever(6, 3, 4)
    d = p.dims
    nn = d.n_nodes
    assert p.fixed.sum() == 3 * (d.ny + 1) * (d.nz + 1)
    for k in range(d.nz + 1):
        for j in range(d.ny + 1):
            n = d.node(0, j, k)
            assert all(p.fixed[c * nn + n] for c in range(3))
    assert np.isclose(p.f.sum(), -1.0)
    assert np.allclose(p.f[: 2 * nn], 0.0)
    fz = p.f[2 * nn:]
    loaded = np.nonzero(fz)[0]
    assert set(loaded) == {d.node(d.nx, j, 0) for j in range(d.ny + 1)}
    assert np.isclose(fz[d.node(d.nx, 0, 0)], 0.5 * fz[d.node(d.nx, 1, 0)])


def test_mbb_supports_and_load():
    p = P.mbb_block(8, 4, 3)
    d = p.dims
    nn = d.n_nodes
    assert np.isclose(p.f.sum(), -1.0)
    assert p.fixed[:nn].sum() == (d.ny + 1) * (d.nz + 1)          # u_x on x = 0
    assert p.fixed[nn:2 * nn].sum() == (d.nx + 1) * (d.nz + 1)    # u_y on y = 0
    assert p.fixed[2 * nn:].sum() == d.ny + 1                      # u_z on the pin line
    top = [d.node(i, j, d.nz) for j in range(d.ny + 1) for i in range(d.nx + 1)]
    assert np.isclose(p.f[2 * nn + np.array(top)].sum(), -1.0)


def test_bumpy_field_is_seeded_and_bounded():
    d = P.GridDims(20, 10, 8)
    a = P.bumpy_field(d, 3)
    b = P.bumpy_field(d, 3)
    c = P.bumpy_field(d, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.05 and a.max() <= 1.0 and a.shape == (d.n_el,)


def test_batch_generator_ranges():
    probs = P.uneven_cantilever_batch(seed=1, count=16)
    assert len(probs) == 16
    for p in probs:
        d = p.dims
        assert 16 <= d.nx <= 64 and 16 <= d.ny <= 32 and 16 <= d.nz <= 32
        assert 0.2 <= p.volfrac <= 0.5 and 1.2 <= p.rmin <= 2.0
        assert np.isclose(p.f.sum(), -1.0) and np.count_nonzero(p.f) == 1


def test_served_requests_are_seeded_and_shaped():
    a = [P.served_request(7, i) for i in range(20)]
    b = [P.served_request(7, i) for i in range(20)]
    for p, q in zip(a, b):
        d = p.dims
        assert d.nx == 2 * d.ny == 2 * d.nz and 12 <= d.ny <= 64
        assert np.array_equal(p.z0, q.z0) and np.array_equal(p.f, q.f)
        assert abs(p.f.sum() + 1.0) <= 1e-12
        assert 0.05 <= p.z0.min() and p.z0.max() <= 1.0
    assert len({p.dims.ny for p in a}) > 5
