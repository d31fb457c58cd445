"""Checks of one library gradient + OC step on grids too large for the oracle's solve.

The oracle evaluates everything but the solve at any size in seconds (filter, product,
sensitivity, filter adjoint, OC), so those are compared element by element; the solve is
checked through properties that hold at any size, with the oracle's FP64 operator:

* residual: for the float displacement u the library returns, ||f - K u|| is at most the
  solver's own residual (target rtol) plus the rounding of u to float,
  2^-24 || |K| |u| || (elementwise |K_ij| |u_j| summed);
* compliance: the library's FP64 f^T u against the oracle's sum on the same u;
* energy: u^T K u = f^T u - u^T r holds in FP64, and u^T r is near zero (a CG residual is
  orthogonal to the Krylov space its iterate lies in).
"""
import os

import numpy as np

from oracle import fem, oc

U32 = 2.0 ** -24
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(fname):
    """(scalars, element indices, dc/dz values) of a full-size oracle golden
    (tests/golden/make_fullsize_goldens.py writes them)."""
    scal, idx, val = {}, [], []
    with open(os.path.join(GOLDEN, fname)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split()
            if a.isdigit():
                idx.append(int(a))
                val.append(float(b))
            else:
                scal[a] = float(b)
    return scal, np.array(idx, np.int64), np.array(val)


def check_golden(fname, c, dcdz, n_el):
    """The library's compliance within 1e-5 relative and its dc/dz at the stored elements
    within 1e-4 (guarded by 1e-3 of max |dc/dz|) of the FP64 oracle's exact gradient
    (Jacobi-PCG to a recursive residual of 1e-12; its true residual, recomputed with the
    oracle's operator and stored, is at most 1e-9, three orders below the library's 1e-6
    target).  Returns (compliance error, dc/dz error)."""
    scal, idx, ref = load_golden(fname)
    assert int(scal["n_el"]) == n_el and scal["true_rel_res"] <= 1e-9
    ec = abs(c / scal["compliance"] - 1.0)
    den = np.maximum(np.abs(ref), 1e-3 * scal["max_abs_dcdz"])
    ed = float(np.max(np.abs(dcdz[idx] - ref) / den))
    assert ec <= 1e-5, ec
    assert ed <= 1e-4, ed
    return ec, ed


def guarded_rel(x, ref):
    """max |x - ref| / max(|ref|, 1e-3 max|ref|), elementwise, then max."""
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(x - ref) / den))


def check_solve(p, m, z, u, c, rtol=1e-6):
    """u solves the oracle's K(P z) u = f to rtol (plus float rounding of u); c = f^T u."""
    E = m.modulus(m.filter(z))
    free = ~m.fixed
    assert np.all(u[m.fixed] == 0.0)
    Ku = m.apply(E, u)
    r = np.where(free, p.f - Ku, 0.0)
    absKu = np.where(free, fem.apply_elementwise(m.nx, m.ny, m.nz, E, p.h, np.abs(m.K0),
                                                 np.abs(u), m.edof), 0.0)
    fn = np.linalg.norm(p.f)
    rn = np.linalg.norm(r)
    assert rn <= 2 * rtol * fn + 1.01 * U32 * np.linalg.norm(absKu), rn / fn
    fu = float(p.f @ u)
    assert abs(c - fu) <= 2 * U32 * float(np.abs(p.f) @ np.abs(u)) + 1e-300
    uKu = float(u @ Ku)
    assert abs(uKu - (fu - float(u @ r))) <= 1e-9 * abs(fu)
    assert abs(uKu / fu - 1.0) <= 1e-5
    return rn / fn


def check_gradient(m, z, u, dcdz, dvdz):
    """dc/dz = P^T dc/drho(P z, u) and dV/dz = P^T v, composed by the oracle in FP64 from
    the library's own (float) u."""
    rho = m.filter(z)
    ref = m.filter_T(m.sensitivity(rho, u))
    err = guarded_rel(dcdz, ref)
    assert err <= 1e-4, err
    assert dcdz.max() <= 1e-6 * np.abs(dcdz).max()
    refv = m.filter_T(m.v)
    assert np.abs(dvdz / refv - 1.0).max() <= 1e-5
    return err


def check_oc(p, m, z, dcdz, dvdz, z_new, change):
    """The OC update on the library's gradient against the oracle's bisection on the same
    inputs; the volume constraint holds when the move limit lets it be met, else every
    element sits at the bound on the side of the constraint."""
    zr, _, ch = oc.oc_update(z, dcdz, dvdz, m.vmax(), p.move)
    assert np.abs(z_new - zr).max() <= 1e-5
    assert abs(change - ch) <= 1e-5
    lo = np.maximum(0.0, z - p.move)
    hi = np.minimum(1.0, z + p.move)
    assert np.all(z_new >= lo - 1e-6) and np.all(z_new <= hi + 1e-6)
    vmax = m.vmax()
    if float(dvdz @ lo) >= vmax:
        assert np.abs(z_new - lo).max() <= 1e-6
    elif float(dvdz @ hi) <= vmax:
        assert np.abs(z_new - hi).max() <= 1e-6
    else:
        assert abs(float(dvdz @ z_new) / vmax - 1.0) <= 1e-5
