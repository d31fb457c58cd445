"""Compliance, sensitivities, filtered gradient and the OC loop, FP64 (oracle; test
infrastructure).

* Objective (Eq. 4): c = f^T u(z).
* Sensitivity (Eq. 5): g_i = -u^T (dK/dz_i) u.  With K = sum_e h E_e(rho_e) K0 and
  E_e = Emin + rho_e^p (E0 - Emin), the derivative with respect to the physical density
  is dc/drho_e = -p rho_e^(p-1) (E0 - Emin) h u_e^T K0 u_e.
* Through the filter rho = P z: dc/dz = P^T dc/drho and dV/dz = P^T v (§III-D), v_e = h^3.
* Loop (Algorithm 1 with every iteration exact): filter, solve, gradient, OC update.
* General objective (Eq. 3): for J = l^T u (a linear functional of the state, dJ/dz = 0
  explicitly), the adjoint lambda solves (dr/du)^T lambda = dJ/du, i.e. K lambda = l
  (K symmetric), and g_i = -lambda^T (dK/dz_i) u; compliance is the case l = f, lambda = u.
"""
from __future__ import annotations

import numpy as np

from . import fem, filt, oc, solve


class Model:
    """Precomputed pieces of one grid: K0, DOF map, filter weight sums."""

    def __init__(self, problem):
        p = problem
        self.p = p
        d = p.dims
        self.nx, self.ny, self.nz = d.nx, d.ny, d.nz
        self.K0 = fem.unit_element_stiffness(p.nu)
        self.edof = fem.element_dofs(d.nx, d.ny, d.nz)
        self.Hs = filt.weight_sums(d.nx, d.ny, d.nz, p.rmin)
        self.fixed = p.fixed.astype(bool)
        self.v = np.full(d.n_el, p.h ** 3)

    # -- pieces ---------------------------------------------------------------------------
    def filter(self, z):
        return filt.filter_forward(self.nx, self.ny, self.nz, self.p.rmin, z, self.Hs)

    def filter_T(self, x):
        return filt.filter_transpose(self.nx, self.ny, self.nz, self.p.rmin, x, self.Hs)

    def modulus(self, rho):
        p = self.p
        return fem.simp_modulus(rho, p.E0, p.Emin, p.penal)

    def apply(self, E, x):
        """K_ff-restricted product on full DOF vectors (fixed entries zero)."""
        free = ~self.fixed
        y = fem.apply_elementwise(self.nx, self.ny, self.nz, E, self.p.h, self.K0,
                                  np.where(free, x, 0.0), self.edof)
        return np.where(free, y, 0.0)

    def solve(self, E, method="auto", tol=1e-12, maxit=200000):
        """u with K_ff u_f = f_f; returns (u, iterations or 0 for direct, rel. residual)."""
        p = self.p
        ndof = p.dims.n_dof
        if method == "auto":
            method = "direct" if ndof <= 60000 else "pcg"
        if method == "direct":
            K = fem.assemble(self.nx, self.ny, self.nz, E, p.h, self.K0)
            u = solve.solve_direct(K, p.f, self.fixed)
            r = np.where(self.fixed, 0.0, p.f - K @ u)
            return u, 0, float(np.linalg.norm(r) / np.linalg.norm(p.f))
        diag = fem.diagonal_elementwise(self.nx, self.ny, self.nz, E, p.h, self.K0, self.edof)
        return solve.solve_pcg_matfree(
            lambda v: fem.apply_elementwise(self.nx, self.ny, self.nz, E, p.h, self.K0, v,
                                            self.edof),
            diag, p.f, self.fixed, tol, maxit)

    def sensitivity(self, rho, u):
        """dc/drho_e = -p rho^(p-1) (E0 - Emin) h u_e^T K0 u_e  (Eq. 5, SIMP chain rule)."""
        p = self.p
        ce = fem.element_energy(self.nx, self.ny, self.nz, u, self.K0, self.edof)
        return -p.penal * np.power(rho, p.penal - 1.0) * (p.E0 - p.Emin) * p.h * ce

    def gradient(self, z, method="auto", tol=1e-12):
        """One exact-gradient evaluation: returns a dict with rho, E, u, c, dc_drho, dcdz,
        dvdz, iters, rel_res."""
        rho = self.filter(z)
        E = self.modulus(rho)
        u, it, rel = self.solve(E, method, tol)
        c = float(self.p.f @ u)
        dc = self.sensitivity(rho, u)
        return dict(rho=rho, E=E, u=u, c=c, dc_drho=dc, dcdz=self.filter_T(dc),
                    dvdz=self.filter_T(self.v), iters=it, rel_res=rel)

    def adjoint_gradient(self, z, l, method="auto", tol=1e-12):
        """Eq. 3 for J = l^T u: returns a dict with J, u, lam, dJ_drho, dJdz."""
        rho = self.filter(z)
        E = self.modulus(rho)
        u, _, _ = self.solve(E, method, tol)
        l = np.where(self.fixed, 0.0, np.asarray(l, np.float64))
        saved = self.p.f
        try:
            self.p.f = l
            lam, _, _ = self.solve(E, method, tol)
        finally:
            self.p.f = saved
        p = self.p
        be = fem.element_bilinear(self.nx, self.ny, self.nz, lam, u, self.K0, self.edof)
        dj = -p.penal * np.power(rho, p.penal - 1.0) * (p.E0 - p.Emin) * p.h * be
        return dict(J=float(l @ u), u=u, lam=lam, dJ_drho=dj, dJdz=self.filter_T(dj))

    def vmax(self):
        return self.p.volfrac * float(np.sum(self.v))

    def oc_step(self, z, dcdz, dvdz, move=None):
        return oc.oc_update(z, dcdz, dvdz, self.vmax(), self.p.move if move is None else move)

    def run(self, iters, z0=None, method="auto", tol=1e-12):
        """OC loop from z0 (default: the problem's initial design).  Returns (z, history)
        with one dict per iteration: c, change, volume of the filtered design."""
        z = np.array(self.p.z0 if z0 is None else z0, np.float64)
        hist = []
        for _ in range(iters):
            g = self.gradient(z, method, tol)
            z, lam, change = self.oc_step(z, g["dcdz"], g["dvdz"])
            hist.append(dict(c=g["c"], change=change, lam=lam,
                             vol=float(self.v @ g["rho"]), iters=g["iters"]))
        return z, hist
