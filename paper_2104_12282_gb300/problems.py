"""Seeded synthetic inputs for the exact-gradient path of SIMP compliance minimisation.

This module builds the *inputs* of the problem stated in Eq. 4 (§III-D): a structured
hex8 voxel grid, the fixed (Dirichlet) degrees of freedom, the load vector f and design
fields z.  It holds none of the method's arithmetic (no stiffness, solve, filter or
optimality-criteria step).  Both the CUDA library and the FP64 CPU oracle receive the
arrays produced here, so they are the only code the two sides share.

Conventions (interface layout, shared by both sides):

* elements ``e = i + nx*(j + ny*k)`` (x fastest), ``0 <= i < nx`` etc.;
* nodes ``n = i + (nx+1)*(j + (ny+1)*k)``;
* nodal vectors are structure-of-arrays: component ``c`` of node ``n`` is at ``c*N_n + n``;
* node ``(i, j, k)`` sits at ``(i*h, j*h, k*h)``.

Loads are consistent nodal forces of a uniform line or face traction, normalised so the
total force is 1 in the -z direction.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass(frozen=True)
class GridDims:
    nx: int
    ny: int
    nz: int

    @property
    def n_el(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_dof(self) -> int:
        """Three displacement components per hex8 node (the count in Table 1)."""
        return 3 * self.n_nodes

    def node(self, i, j, k):
        return i + (self.nx + 1) * (j + (self.ny + 1) * k)

    def elem(self, i, j, k):
        return i + self.nx * (j + self.ny * k)


@dataclass
class Problem:
    """One compliance-minimisation instance (Eq. 4) on a structured grid."""
    name: str
    dims: GridDims
    h: float
    E0: float
    Emin: float
    nu: float
    penal: float
    rmin: float          # filter radius in element units
    volfrac: float
    fixed: np.ndarray    # uint8[3*N_n], 1 = displacement fixed to 0 (SoA order)
    f: np.ndarray        # float64[3*N_n] load vector (SoA order)
    move: float = 0.2
    z0: Optional[np.ndarray] = None   # float64[N_el] initial design
    meta: dict = field(default_factory=dict)

    @property
    def n_el(self):
        return self.dims.n_el


def _node_grid(d: GridDims):
    k, j, i = np.meshgrid(np.arange(d.nz + 1), np.arange(d.ny + 1), np.arange(d.nx + 1),
                          indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def _edge_weights(n: int) -> np.ndarray:
    """Trapezoid weights of n equal segments (ends 1/2): consistent nodal load of a
    uniform line traction on linear elements."""
    w = np.ones(n + 1)
    w[0] = w[-1] = 0.5
    return w


def cantilever(nx: int, ny: int, nz: int, *, h: float = 1.0, volfrac: float = 0.3,
               rmin: float = 1.5, E0: float = 1.0, Emin: float = 1e-9, nu: float = 0.3,
               penal: float = 3.0, move: float = 0.2) -> Problem:
    """Cantilever of §IV: face x=0 clamped, unit downward line load along the lower edge
    (z=0) of the face x=nx, consistent nodal weights (end nodes 1/2), total force 1."""
    d = GridDims(nx, ny, nz)
    nn = d.n_nodes
    i, j, k = _node_grid(d)
    fixed = np.zeros(3 * nn, np.uint8)
    clamp = np.nonzero(i == 0)[0]
    for c in range(3):
        fixed[c * nn + clamp] = 1
    f = np.zeros(3 * nn)
    wy = _edge_weights(ny) / ny
    for jj in range(ny + 1):
        f[2 * nn + d.node(nx, jj, 0)] = -wy[jj]
    z0 = np.full(d.n_el, volfrac)
    return Problem("cantilever", d, h, E0, Emin, nu, penal, rmin, volfrac, fixed, f, move, z0)


def mbb_block(nx: int, ny: int, nz: int, *, h: float = 1.0, volfrac: float = 0.12,
              rmin: float = 2.5, E0: float = 1.0, Emin: float = 1e-9, nu: float = 0.3,
              penal: float = 3.0, move: float = 0.2) -> Problem:
    """Quarter bridge / MBB-type block: symmetry planes x=0 (u_x=0) and y=0 (u_y=0), a pin
    line (u_z=0) along x=nx, z=0, and a uniform traction on the top face z=nz totalling 1
    in -z with consistent bilinear nodal weights."""
    d = GridDims(nx, ny, nz)
    nn = d.n_nodes
    i, j, k = _node_grid(d)
    fixed = np.zeros(3 * nn, np.uint8)
    fixed[0 * nn + np.nonzero(i == 0)[0]] = 1
    fixed[1 * nn + np.nonzero(j == 0)[0]] = 1
    fixed[2 * nn + np.nonzero((i == nx) & (k == 0))[0]] = 1
    f = np.zeros(3 * nn)
    wx = _edge_weights(nx) / nx
    wy = _edge_weights(ny) / ny
    top = np.nonzero(k == nz)[0]
    f[2 * nn + top] = -(wx[i[top]] * wy[j[top]])
    z0 = np.full(d.n_el, volfrac)
    return Problem("mbb_block", d, h, E0, Emin, nu, penal, rmin, volfrac, fixed, f, move, z0)


def coarse_problem(p: Problem, nb: int) -> Problem:
    """The same problem (supports, load, material) on the coarse grid of the two-scale
    scheme: ceil(n / N_B) elements per axis of edge N_B h.  Only the cantilever and the
    MBB-type block are defined here; their loads are resolution independent (total 1)."""
    d = p.dims
    dims = (-(-d.nx // nb), -(-d.ny // nb), -(-d.nz // nb))
    kw = dict(h=p.h * nb, volfrac=p.volfrac, rmin=p.rmin, E0=p.E0, Emin=p.Emin, nu=p.nu,
              penal=p.penal, move=p.move)
    if p.name == "cantilever":
        q = cantilever(*dims, **kw)
    elif p.name == "mbb_block":
        q = mbb_block(*dims, **kw)
    else:
        raise ValueError(f"no coarse definition for problem {p.name!r}")
    q.meta["block_size"] = nb
    q.meta["fine"] = (d.nx, d.ny, d.nz)
    return q


def bumpy_field(d: GridDims, seed: int, *, lo: float = 0.05, hi: float = 1.0,
                n_bumps: int = 8, amp: float = 0.3, sigma=(4.0, 16.0)) -> np.ndarray:
    """Design field: U[lo, hi] noise plus smooth Gaussian bumps, clipped to [lo, hi].

    z = clip(U[lo,hi] + sum_k a_k exp(-|x - c_k|^2 / (2 s_k^2)), lo, hi), a_k ~ U[-amp, amp],
    s_k ~ U[sigma], c_k uniform in the box (element units).  float64[N_el]."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(lo, hi, size=d.n_el)
    kk, jj, ii = np.meshgrid(np.arange(d.nz) + 0.5, np.arange(d.ny) + 0.5,
                             np.arange(d.nx) + 0.5, indexing="ij")
    X = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    for _ in range(n_bumps):
        a = rng.uniform(-amp, amp)
        s = rng.uniform(*sigma)
        c = rng.uniform([0, 0, 0], [d.nx, d.ny, d.nz])
        r2 = np.sum((X - c) ** 2, axis=1)
        z += a * np.exp(-r2 / (2 * s * s))
    return np.clip(z, lo, hi)


def random_field(d: GridDims, seed: int, lo: float = 0.05, hi: float = 1.0) -> np.ndarray:
    """Plain U[lo, hi] field, float64[N_el]."""
    return np.random.default_rng(seed).uniform(lo, hi, size=d.n_el)


def random_nodal(d: GridDims, seed: int, fixed: Optional[np.ndarray] = None) -> np.ndarray:
    """U[-1, 1] nodal vector float64[3*N_n], zero where ``fixed`` is set."""
    x = np.random.default_rng(seed).uniform(-1.0, 1.0, size=d.n_dof)
    if fixed is not None:
        x[fixed.astype(bool)] = 0.0
    return x


def random_sensitivity(d: GridDims, seed: int) -> np.ndarray:
    """A negative compliance-like sensitivity field (float64[N_el]), for OC-step inputs."""
    rng = np.random.default_rng(seed)
    return -np.exp(rng.uniform(-6.0, 0.0, size=d.n_el))


# ---------------------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------------------

def cantilever_24x12x12() -> Problem:
    """24x12x12 cantilever, FP64, volfrac 0.3, rmin 1.5, uniform start, 10 OC iterations."""
    p = cantilever(24, 12, 12, volfrac=0.3, rmin=1.5)
    p.meta["oc_iters"] = 10
    return p


def cantilever_96x48x48() -> Problem:
    """96x48x48 cantilever, FP32 GMG-PCG (4 levels), rel. residual 1e-6, 50 OC iterations."""
    p = cantilever(96, 48, 48, volfrac=0.3, rmin=1.5)
    p.meta["oc_iters"] = 50
    p.meta["mg_levels"] = 4
    return p


def mbb_192x96x76(seed: int = 0) -> Problem:
    """192x96x76 MBB-type block (1,400,832 design variables), volfrac 0.12, rmin 2.5,
    design field from ``bumpy_field``."""
    p = mbb_block(192, 96, 76, volfrac=0.12, rmin=2.5)
    p.z0 = bumpy_field(p.dims, seed)
    p.meta["seed"] = seed
    return p


def uneven_cantilever_batch(seed: int = 0, count: int = 64) -> List[Problem]:
    """Batch of uneven cantilevers: nx ~ U{16..64}, ny, nz ~ U{16..32}; one loaded node
    drawn uniformly on the face x=nx (unit -z force); volfrac ~ U[0.2, 0.5];
    rmin ~ U[1.2, 2.0]; the face x=0 clamped; uniform start at volfrac."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        nx = int(rng.integers(16, 65))
        ny = int(rng.integers(16, 33))
        nz = int(rng.integers(16, 33))
        vf = float(rng.uniform(0.2, 0.5))
        rm = float(rng.uniform(1.2, 2.0))
        p = cantilever(nx, ny, nz, volfrac=vf, rmin=rm)
        d = p.dims
        p.f[:] = 0.0
        jj = int(rng.integers(0, ny + 1))
        kk = int(rng.integers(0, nz + 1))
        p.f[2 * d.n_nodes + d.node(nx, jj, kk)] = -1.0
        p.name = f"cantilever_{nx}x{ny}x{nz}_b{b}"
        out.append(p)
    return out


def served_request(seed: int, index: int, n_range=(12, 64)) -> Problem:
    """One request of a served stream: a 2n x n x n domain, n ~ U{n_range}, either the
    cantilever with one loaded node drawn on the face x = nx or the MBB-type block; volume
    fraction ~ U[0.1, 0.4], rmin ~ U[1.2, 2.5]; design field U[0.05, 1]."""
    rng = np.random.default_rng([seed, index])
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    vf = float(rng.uniform(0.1, 0.4))
    rm = float(rng.uniform(1.2, 2.5))
    if rng.uniform() < 0.5:
        p = cantilever(2 * n, n, n, volfrac=vf, rmin=rm)
        d = p.dims
        p.f[:] = 0.0
        jj = int(rng.integers(0, n + 1))
        kk = int(rng.integers(0, n + 1))
        p.f[2 * d.n_nodes + d.node(2 * n, jj, kk)] = -1.0
        p.name = f"served_cantilever_{index}"
    else:
        p = mbb_block(2 * n, n, n, volfrac=vf, rmin=rm)
        p.name = f"served_mbb_{index}"
    p.z0 = random_field(p.dims, int(rng.integers(0, 2 ** 31)), 0.05, 1.0)
    p.meta["request"] = index
    return p


def table1_meshes():
    """Cantilever meshes of Table 1 on a 2:1:1 domain: (fine dims, N_B)."""
    return [((70, 35, 35), 5), ((100, 50, 50), 5), ((180, 90, 90), 5)]
