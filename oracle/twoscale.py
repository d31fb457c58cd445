"""Two-scale coarse-graining and the coarse-scale state (oracle; test infrastructure).

§III-C and §III-D: the design variables are grouped by location into N_B x N_B x N_B blocks
of elements; each component of the coarse design z_C is the average of z over one block,
and the coarse-scale constraints r_C(z_C, u_C) = K_C(z_C) u_C - f_C = 0 are solved for u_C
(Algorithm 1, the two steps at the top of every iteration).  The coarse stiffness is the
same hex8 SIMP stiffness on the coarse grid (element edge N_B h) with moduli
E_e = Emin + z_C,e^p (E0 - Emin) taken from z_C directly: the paper applies the density
filter to the fine design only.  f_C is the problem's load discretised on the coarse grid.

Reading for grids that N_B does not divide (the paper's meshes are divisible): the last
block along an axis holds the remaining elements and z_C is the mean over the elements it
holds, so the coarse grid has ceil(n / N_B) elements along that axis.
"""
from __future__ import annotations

import numpy as np

from . import topopt


def coarse_dims(nx: int, ny: int, nz: int, nb: int):
    """Elements per axis of the coarse grid: ceil(n / N_B)."""
    return (-(-nx // nb), -(-ny // nb), -(-nz // nb))


def coarse_grain(nx: int, ny: int, nz: int, nb: int, z):
    """z_C[I + cx (J + cy K)] = mean of z over block (I, J, K) (x-fastest element order)."""
    cx, cy, cz = coarse_dims(nx, ny, nz, nb)
    Z = np.asarray(z, np.float64).reshape(nz, ny, nx)
    zc = np.empty(cx * cy * cz)
    for K in range(cz):
        for J in range(cy):
            for I in range(cx):
                blk = Z[K * nb:(K + 1) * nb, J * nb:(J + 1) * nb, I * nb:(I + 1) * nb]
                zc[I + cx * (J + cy * K)] = blk.mean()
    return zc


def coarse_state(coarse_problem, zc, method="auto", tol=1e-12):
    """u_C with K_C(z_C) u_C = f_C on the coarse problem (no filter on z_C).  Returns
    (u_C, c_C = f_C^T u_C)."""
    m = topopt.Model(coarse_problem)
    u, _, _ = m.solve(m.modulus(np.asarray(zc, np.float64)), method, tol)
    return u, float(coarse_problem.f @ u)
