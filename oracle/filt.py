"""Density filter P (oracle; test infrastructure).

Eq. 4 constrains v^T P z, where P is the density filter matrix (§III-D); the filtered
(physical) densities are rho = P z.  The paper gives no formula for P beyond its name and
the radius R.  Reading used here: linear cone weights H_ij = max(0, rmin - |x_i - x_j|)
between element centroids (element units), rows normalised by Hs_i = sum_j H_ij over
neighbours inside the domain, so P = diag(1/Hs) H.  H is symmetric, hence
P^T x = H (x / Hs); the volume gradient of §III-D is P^T v.

Two equivalent evaluations, cross-checked in the tests: an explicit sparse H (small
grids) and a shifted-array stencil (any size).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def stencil_offsets(rmin: float):
    """All (di, dj, dk, w) with w = rmin - sqrt(di^2 + dj^2 + dk^2) > 0."""
    R = int(np.ceil(rmin)) - 1
    out = []
    for dk in range(-R, R + 1):
        for dj in range(-R, R + 1):
            for di in range(-R, R + 1):
                w = rmin - np.sqrt(di * di + dj * dj + dk * dk)
                if w > 0.0:
                    out.append((di, dj, dk, w))
    return out


def filter_matrix(nx: int, ny: int, nz: int, rmin: float):
    """Explicit (H, Hs): H sparse symmetric N_el x N_el, Hs = H 1."""
    n = nx * ny * nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    rows, cols, vals = [], [], []
    for di, dj, dk, w in stencil_offsets(rmin):
        ii, jj, kk = i + di, j + dj, k + dk
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
        src = np.nonzero(ok)[0]
        dst = ii[ok] + nx * (jj[ok] + ny * kk[ok])
        rows.append(src)
        cols.append(dst)
        vals.append(np.full(src.size, w))
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    Hs = np.asarray(H.sum(axis=1)).ravel()
    return H, Hs


def _shift_accumulate(nx, ny, nz, x, rmin):
    """sum_j H_ij x_j for all i via shifted 3-D arrays (no matrix)."""
    X = x.reshape(nz, ny, nx)
    out = np.zeros_like(X)
    for di, dj, dk, w in stencil_offsets(rmin):
        if abs(di) >= nx or abs(dj) >= ny or abs(dk) >= nz:
            continue  # no pair of in-domain elements at this offset
        # out[k, j, i] += w * X[k+dk, j+dj, i+di] where in range
        ks = slice(max(0, -dk), nz - max(0, dk))
        js = slice(max(0, -dj), ny - max(0, dj))
        is_ = slice(max(0, -di), nx - max(0, di))
        ks2 = slice(max(0, dk), nz - max(0, -dk))
        js2 = slice(max(0, dj), ny - max(0, -dj))
        is2 = slice(max(0, di), nx - max(0, -di))
        out[ks, js, is_] += w * X[ks2, js2, is2]
    return out.ravel()


def weight_sums(nx: int, ny: int, nz: int, rmin: float) -> np.ndarray:
    """Hs = H 1, truncated at the domain boundary."""
    return _shift_accumulate(nx, ny, nz, np.ones(nx * ny * nz), rmin)


def filter_forward(nx, ny, nz, rmin, z, Hs=None):
    """rho = P z = (H z) / Hs."""
    if Hs is None:
        Hs = weight_sums(nx, ny, nz, rmin)
    return _shift_accumulate(nx, ny, nz, np.asarray(z, np.float64), rmin) / Hs


def filter_transpose(nx, ny, nz, rmin, x, Hs=None):
    """P^T x = H (x / Hs)."""
    if Hs is None:
        Hs = weight_sums(nx, ny, nz, rmin)
    return _shift_accumulate(nx, ny, nz, np.asarray(x, np.float64) / Hs, rmin)


def filter_forward_at(nx, ny, nz, rmin, z, elems):
    """rho_e = (H z)_e / Hs_e for selected element indices only, one element at a time
    (used to spot-check outputs on grids too large for a full evaluation)."""
    z = np.asarray(z, np.float64)
    offs = stencil_offsets(rmin)
    out = np.empty(len(elems))
    for t, e in enumerate(elems):
        i = e % nx
        j = (e // nx) % ny
        k = e // (nx * ny)
        num = 0.0
        den = 0.0
        for di, dj, dk, w in offs:
            ii, jj, kk = i + di, j + dj, k + dk
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                num += w * z[ii + nx * (jj + ny * kk)]
                den += w
        out[t] = num / den
    return out
