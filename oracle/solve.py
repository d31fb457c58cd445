"""State solve K_ff u_f = f_f, FP64 (oracle; test infrastructure).

§III-D: u(z) is defined by K(z) u - f = 0; the paper's standard optimizer solves it by PCG
with a Jacobi preconditioner (§IV, "Competitor method").  Fixed DOFs carry u = 0 and are
removed from the system.  Two solvers, cross-checked in the tests:

* ``solve_direct``  -- sparse LU of K_ff (small grids, exact up to rounding);
* ``pcg_jacobi``    -- textbook Jacobi-preconditioned CG on any operator, run to a
                       relative residual of 1e-12 for parity use.
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve_direct(K: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """u with u[fixed] = 0 and K_ff u_f = f_f, by sparse LU."""
    free = ~np.asarray(fixed, dtype=bool)
    Kff = K[free][:, free].tocsc()
    u = np.zeros(K.shape[0])
    u[free] = spla.spsolve(Kff, f[free])
    return u


def pcg_jacobi(apply: Callable[[np.ndarray], np.ndarray], diag: np.ndarray, b: np.ndarray,
               tol: float = 1e-12, maxit: int = 100000, x0: np.ndarray | None = None
               ) -> Tuple[np.ndarray, int, float]:
    """Preconditioned CG with M = diag(A): returns (x, iterations, ||b - A x|| / ||b||)
    where the residual is the recursively updated one."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply(x) if x0 is not None else b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    dinv = 1.0 / diag
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / bnorm
    while rel > tol and it < maxit:
        q = apply(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        rel = np.linalg.norm(r) / bnorm
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, rel


def solve_pcg_csr(K: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray, tol: float = 1e-12,
                  maxit: int = 100000) -> Tuple[np.ndarray, int, float]:
    """u with u[fixed] = 0 from Jacobi-PCG on the assembled K_ff."""
    free = ~np.asarray(fixed, dtype=bool)
    Kff = K[free][:, free].tocsr()
    uf, it, rel = pcg_jacobi(lambda v: Kff @ v, Kff.diagonal(), f[free], tol, maxit)
    u = np.zeros(K.shape[0])
    u[free] = uf
    return u, it, rel


def solve_pcg_matfree(apply_full: Callable[[np.ndarray], np.ndarray], diag_full: np.ndarray,
                      f: np.ndarray, fixed: np.ndarray, tol: float = 1e-12,
                      maxit: int = 100000) -> Tuple[np.ndarray, int, float]:
    """Same as ``solve_pcg_csr`` with K applied element by element on the full DOF
    vector; fixed DOFs are zeroed before and after each product (K_ff restriction)."""
    free = ~np.asarray(fixed, dtype=bool)

    def apply(v):
        y = apply_full(np.where(free, v, 0.0))
        return np.where(free, y, 0.0)

    diag = np.where(free, diag_full, 1.0)
    b = np.where(free, f, 0.0)
    return pcg_jacobi(apply, diag, b, tol, maxit)
