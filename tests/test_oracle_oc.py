"""Pins of the oracle's optimality-criteria update (no GPU)."""
import numpy as np

from oracle import oc


def test_closed_form_multiplier_when_no_bound_is_active():
    """With no clamp active, V(lam) = sum w z sqrt(-dc/(lam w)) = Vmax gives
    lam* = (sum z sqrt(-dc w))^2 / Vmax^2 exactly."""
    rng = np.random.default_rng(0)
    n = 500
    z = rng.uniform(0.4, 0.6, n)
    w = rng.uniform(0.5, 1.5, n)
    dc = -w * rng.uniform(0.9, 1.1, n)      # -dc/w ~ 1: z_new ~ z / sqrt(lam)
    vmax = 0.97 * np.sum(w * z)
    lam_star = (np.sum(z * np.sqrt(-dc * w)) / vmax) ** 2
    znew, lam, change = oc.oc_update(z, dc, w, vmax, move=1.0)
    assert abs(lam / lam_star - 1.0) <= 1e-9
    expect = z * np.sqrt(-dc / (lam_star * w))
    assert np.all((expect > 0) & (expect < 1))
    assert np.abs(znew - expect).max() <= 1e-9
    assert np.isclose(change, np.abs(expect - z).max(), rtol=1e-8)


def test_volume_bounds_move_limit_and_scaling():
    rng = np.random.default_rng(1)
    n = 2000
    z = rng.uniform(0.0, 1.0, n)
    w = rng.uniform(0.2, 1.0, n)
    dc = -np.exp(rng.uniform(-5, 1, n))
    vmax = 0.4 * w.sum()
    move = 0.2
    znew, lam, change = oc.oc_update(z, dc, w, vmax, move)
    assert abs(np.sum(w * znew) - vmax) <= 1e-8 * vmax
    assert np.all(znew >= 0) and np.all(znew <= 1)
    assert np.all(np.abs(znew - z) <= move + 1e-15)
    z2, lam2, _ = oc.oc_update(z, 7.5 * dc, w, vmax, move)
    assert np.isclose(lam2, 7.5 * lam, rtol=1e-8)
    assert np.abs(z2 - znew).max() <= 1e-8


def test_uniform_input_gives_uniform_output():
    n = 300
    z = np.full(n, 0.3)
    znew, _, _ = oc.oc_update(z, np.full(n, -2.0), np.full(n, 1.0), 0.35 * n, 0.2)
    assert np.ptp(znew) == 0.0 and np.isclose(znew[0], 0.35, rtol=1e-9)


def test_infeasible_target_returns_lower_bounds():
    """If even the lower move limits exceed V_max the multiplier runs to its cap and every
    entry sits on max(0, z - move)."""
    rng = np.random.default_rng(2)
    z = rng.uniform(0.5, 1.0, 400)
    w = np.ones_like(z)
    dc = -rng.uniform(0.1, 1.0, z.size)
    znew, lam, _ = oc.oc_update(z, dc, w, 0.05 * z.size, 0.2)
    assert lam > 1e29
    assert np.abs(znew - np.maximum(0.0, z - 0.2)).max() <= 1e-12


def test_zero_or_positive_sensitivity_goes_to_lower_bound():
    z = np.array([0.5, 0.5, 0.5, 0.5])
    dc = np.array([0.0, 1.0, -1.0, -1.0])
    w = np.ones(4)
    znew, _, _ = oc.oc_update(z, dc, w, 1.6, 0.2)
    assert znew[0] == 0.3 and znew[1] == 0.3
    assert np.isclose(znew.sum(), 1.6, rtol=1e-9)


def test_inactive_volume_bound_gives_upper_bounds():
    """If every entry at its upper move limit still stays below V_max, the multiplier runs
    to its floor 2^-100 and the update is min(1, z + move) (zero sensitivity excepted)."""
    z = np.array([0.25, 0.6, 0.9])
    dc = np.array([-0.4, -1.0, -2.0])
    w = np.ones(3)
    znew, lam, _ = oc.oc_update(z, dc, w, 2.9, 0.2)
    assert lam <= 2.0 ** -100
    assert np.allclose(znew, np.minimum(1.0, z + 0.2), rtol=0, atol=1e-15)
    znew1, _, _ = oc.oc_update(z[:1], dc[:1], w[:1], 0.5, 0.2)
    assert np.isclose(znew1[0], 0.45)
