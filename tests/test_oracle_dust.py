"""Pins of the oracle's dust source update and CFL step (Sec. 3.1) against
facts that do not depend on its code: a Keplerian orbit is an equilibrium of
the sources, a grain at rest above the mid-plane falls under the vertical
gravity, the drag update solves backward Euler for dv/dt = -(v - v_g)/t_s,
tightly coupled grains take the gas velocity, mass and (without drag)
angular momentum are untouched, and the CFL step of uniform grids has its
closed form."""
import math

import numpy as np
import pytest

from oracle import dust

G_M = 6.674e-8 * 1.989e33
AU = 1.496e13


def setup(n_s=3, n_c=5, seed=0):
    rng = np.random.default_rng(seed)
    R = AU * rng.uniform(5, 50, n_c)
    Z = R * rng.uniform(0.0, 0.1, n_c)
    rho_g = 10.0 ** rng.uniform(-14, -11, n_c)
    c_s = rng.uniform(2e4, 8e4, n_c)
    a = 10.0 ** rng.uniform(-5, 0, n_s)
    return R, Z, rho_g, c_s, a


def conserved(P, R):
    return np.stack([P[0], P[0] * P[1], P[0] * P[2] * R[None, :], P[0] * P[3]])


def test_keplerian_orbit_is_an_equilibrium():
    R, Z, rho_g, c_s, a = setup()
    Z = np.zeros_like(Z)
    Om = np.sqrt(G_M / R ** 3)
    n_s = a.size
    P = np.zeros((4, n_s, R.size))
    P[0] = 1e-15
    P[2] = Om * R
    v_g = np.stack([np.zeros_like(R), Om * R, np.zeros_like(R)])
    Q = conserved(P, R)
    out = dust.source_update(Q, P, 3e8, R, Z, rho_g, c_s, v_g, a, 1.6, G_M)
    # v_phi^2 / R and Omega^2 R cancel to rounding: velocities move by ~1e-16
    # of h Omega^2 R
    scale = P[0] * Om * R
    assert np.all(np.abs(out - Q) <= 1e-12 * np.stack([scale, scale, scale * R, scale]))


def test_vertical_fall_without_drag():
    """Huge grains in thin gas (t_s >> h): a grain at rest at height Z gains
    v_Z = -h Omega^2 Z, Omega^2 = G M / (R^2 + Z^2)^(3/2), to O(h / t_s)."""
    R = np.array([10 * AU]); Z = np.array([AU])
    rho_g, c_s, a = np.array([1e-20]), np.array([3e4]), np.array([100.0])
    P = np.zeros((4, 1, 1)); P[0] = 1e-18
    h = 1e5
    out = dust.source_update(conserved(P, R), P, h, R, Z, rho_g, c_s, np.zeros((3, 1)), a, 1.6, G_M)
    Om2 = G_M / (R[0] ** 2 + Z[0] ** 2) ** 1.5
    ts = 1.6 * 100.0 / (1e-20 * math.sqrt(8 / math.pi) * 3e4)
    assert out[3, 0, 0] / P[0, 0, 0] == pytest.approx(-h * Om2 * Z[0], rel=2 * h / ts + 1e-12)
    assert out[1, 0, 0] / P[0, 0, 0] == pytest.approx(-h * Om2 * R[0], rel=2 * h / ts + 1e-12)


def test_drag_is_backward_euler_and_couples_small_grains():
    R, Z, rho_g, c_s, a = setup(seed=2)
    rng = np.random.default_rng(3)
    n_s, n_c = a.size, R.size
    P = np.zeros((4, n_s, n_c))
    P[0] = 1e-14
    P[1:] = rng.normal(0, 1e3, (3, n_s, n_c))
    P[2] = 0.0                                  # no v_phi: no curvature source
    v_g = rng.normal(0, 1e3, (3, n_c))
    GM0 = 0.0                                   # no gravity: drag alone
    h = 1e7
    out = dust.source_update(conserved(P, R), P, h, R, Z, rho_g, c_s, v_g, a, 1.6, GM0)
    v_new = np.stack([out[1] / out[0], out[2] / (out[0] * R), out[3] / out[0]])
    v_old = P[1:]
    vth = math.sqrt(8 / math.pi) * c_s
    ts = 1.6 * a[:, None] / (rho_g[None, :] * vth[None, :])
    # (v' - v) / h = -(v' - v_g) / t_s
    res = (v_new - v_old) / h + (v_new - v_g[:, None, :]) / ts[None]
    scale = np.abs(v_old - v_g[:, None, :]) / np.minimum(ts, h)[None] + 1e-300
    assert np.all(np.abs(res) <= 1e-12 * scale)
    assert np.array_equal(out[0], P[0])
    # t_s -> 0: the gas velocity
    tiny = dust.source_update(conserved(P, R), P, h, R, Z, rho_g * 1e30, c_s, v_g, a, 1.6, GM0)
    assert np.allclose(tiny[3] / tiny[0], v_g[2][None, :], rtol=1e-12, atol=1e-9)


def test_angular_momentum_without_azimuthal_drag():
    R, Z, rho_g, c_s, a = setup(seed=4)
    rng = np.random.default_rng(5)
    P = np.zeros((4, a.size, R.size)); P[0] = 1e-13
    P[1:] = rng.normal(0, 1e4, (3, a.size, R.size))
    v_g = np.stack([np.zeros_like(R), P[2, 0], np.zeros_like(R)])
    P[2] = P[2, 0][None, :]                     # every species co-rotates with the gas
    out = dust.source_update(conserved(P, R), P, 1e8, R, Z, rho_g, c_s, v_g, a, 1.6, G_M)
    assert np.allclose(out[2], conserved(P, R)[2], rtol=1e-14, atol=0)


def test_cfl_closed_forms():
    n_c = 7
    dR = np.full(n_c, 2.0); dZ = np.full(n_c, 3.0)
    vR = np.full((2, n_c), 5.0); vZ = np.zeros((2, n_c))
    # advection-limited: 0.4 x 2 / 5
    assert dust.cfl_dt(vR, vZ, dR, dZ, np.full(n_c, 1e-9), np.ones(2)) == pytest.approx(0.16)
    # diffusion-limited, Sc = 2 on one species: 0.2 x 2^2 x 1 / 10
    assert dust.cfl_dt(np.zeros((2, n_c)), vZ, dR, dZ, np.full(n_c, 10.0),
                       np.array([1.0, 2.0])) == pytest.approx(0.08)
    # one fast cell sets it
    vR[1, 3] = -100.0
    assert dust.cfl_dt(vR, vZ, dR, dZ, np.full(n_c, 1e-9), np.ones(2)) == pytest.approx(0.4 * 2 / 100)
