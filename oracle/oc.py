"""Optimality-criteria design update (oracle; test infrastructure).

§III-D updates z with the optimality criteria (OC) method, the standard optimizer for
Eq. 4; Algorithm 1 applies it once per iteration ("update z with g").  The paper does not
state its constants.  Reading used here (the usual heuristic OC fixed point):

    B_e(lam)   = max(-dc/dz_e, 0) / (lam * dV/dz_e)
    z_new,e    = clamp(z_e * B_e(lam)^eta, max(0, z_e - m), min(1, z_e + m)),  eta = 1/2
    V(lam)     = sum_e dV/dz_e * z_new,e          (= v^T P z_new, the constraint of Eq. 4)

with lam chosen by bisection so that V(lam) = V_max: l1 = 0, l2 = 1 doubled (at most 100
times) until V(l2) <= V_max, then halving until (l2 - l1)/(l1 + l2) <= tol; the update is
evaluated at the final midpoint.  The multiplier is confined to [2^-100, 2^100]: if the
volume bound cannot bind (V(lam) <= V_max even as lam -> 0, every entry at its upper move
limit) the halving stops once l2 <= 2^-100; if it cannot be met (V(lam) > V_max at 2^100)
the result sits at the lower move limits.
"""
from __future__ import annotations

import numpy as np


def oc_candidate(z, dcdz, dvdz, lam, move, eta=0.5):
    """z_new at a given multiplier lam."""
    z = np.asarray(z, np.float64)
    lo = np.maximum(0.0, z - move)
    hi = np.minimum(1.0, z + move)
    B = np.maximum(-np.asarray(dcdz, np.float64), 0.0) / (lam * np.asarray(dvdz, np.float64))
    return np.clip(z * np.power(B, eta), lo, hi)


def oc_update(z, dcdz, dvdz, vmax, move=0.2, eta=0.5, tol=1e-10, max_doublings=100):
    """Returns (z_new, lam, change) with change = max |z_new - z|."""
    dvdz = np.asarray(dvdz, np.float64)

    def vol(lam):
        return float(np.sum(dvdz * oc_candidate(z, dcdz, dvdz, lam, move, eta)))

    l1, l2 = 0.0, 1.0
    n = 0
    while vol(l2) > vmax and n < max_doublings:
        l2 *= 2.0
        n += 1
    while (l2 - l1) / (l1 + l2) > tol and l2 > 2.0 ** -100:
        lmid = 0.5 * (l1 + l2)
        if vol(lmid) > vmax:
            l1 = lmid
        else:
            l2 = lmid
    lam = 0.5 * (l1 + l2)
    z_new = oc_candidate(z, dcdz, dvdz, lam, move, eta)
    change = float(np.max(np.abs(z_new - np.asarray(z, np.float64)))) if z_new.size else 0.0
    return z_new, lam, change
