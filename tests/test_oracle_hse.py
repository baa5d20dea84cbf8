"""Pins of the hydrostatic-equilibrium oracle (Sec. 3.5, Eqs. hedisc, avcs,
heprod, rhonorm) against closed forms that do not depend on its code.
"""
import math

import numpy as np

from paper_2402_18471_b300 import synth
from oracle import hse

AU = synth.CONST["au"]
GM = synth.CONST["G"] * synth.CONST["M_sun"]
K_B, M_H, MU = synth.CONST["k_B"], synth.CONST["m_H"], 2.4


def column(n_Z, T, R=10 * AU, Ztop=0.2 * 10 * AU):
    """One column of n_Z cells, uniform in Z over 0..Ztop at radius R."""
    Ze = np.linspace(0.0, Ztop, n_Z + 1)
    Z = 0.5 * (Ze[1:] + Ze[:-1])[None, :]
    Re = np.array([0.95 * R, 1.05 * R])
    V = 0.5 * (Re[1] ** 2 - Re[0] ** 2) * np.diff(Ze)[None, :]
    return dict(R=np.full((1, n_Z), R), Z=Z, T=np.broadcast_to(T, (1, n_Z)).copy(), V=V, R_edges=Re,
                Sigma_g=np.array([3.0]), mu=MU, m_H=M_H, k_B=K_B, GM=GM)


def test_isothermal_column_telescopes():
    """Constant c_s: the product of Eq. heprod telescopes to
    P_j / P_0 = exp[G M_* / c_s^2 (1/r_j - 1/r_0)]."""
    c = column(40, 30.0)
    rho = hse.hse_rho_gas(**c)[0]
    cs2 = K_B * 30.0 / (MU * M_H)
    r = np.hypot(c["R"][0], c["Z"][0])
    want = np.exp(GM / cs2 * (1.0 / r - 1.0 / r[0]))
    assert np.allclose(rho / rho[0], want, rtol=1e-12, atol=0)


def test_linear_reciprocal_sound_speed_is_integrated_exactly():
    """With 1/c_s^2 = a + b u, u = 1/r, d ln P = G M_* (1/c_s^2) du and the
    mean of Eq. avcs (the trapezoid rule in u) is exact:
    ln(P_j / P_0) = G M_* [a (u_j - u_0) + b (u_j^2 - u_0^2) / 2]."""
    c = column(25, 1.0)
    r = np.hypot(c["R"][0], c["Z"][0])
    u = 1.0 / r
    cs2_0 = K_B * 40.0 / (MU * M_H)
    a = 0.4 / cs2_0
    b = 0.6 / cs2_0 / u[0]                      # 1/c_s^2 = 1/cs2_0 at the mid-plane cell
    inv_cs2 = a + b * u
    c["T"] = (MU * M_H / K_B / inv_cs2)[None, :]
    rho = hse.hse_rho_gas(**c)[0]
    lnP = GM * (a * (u - u[0]) + 0.5 * b * (u ** 2 - u[0] ** 2))
    omega = np.exp(lnP) * inv_cs2
    assert np.allclose(rho / rho[0], omega / omega[0], rtol=1e-12, atol=0)


def test_normalised_to_the_column_mass_and_positive():
    d = synth.make_disc(7, 48, 10, 1e-5, 1e-3, 5.0, 100.0, 1.0)
    inp = synth.hse_inputs(d, t_rise=3.0)
    rho = hse.hse_rho_gas(**inp)
    RdR = 0.5 * (inp["R_edges"][1:] ** 2 - inp["R_edges"][:-1] ** 2)
    assert np.allclose((rho * inp["V"]).sum(1), inp["Sigma_g"] * RdR, rtol=1e-13)
    assert np.all(rho > 0)
    # warmer upper layers hold more gas up there than the isothermal column
    iso = hse.hse_rho_gas(**synth.hse_inputs(d))
    assert np.all(rho[:, -1] > iso[:, -1])


def test_thin_disc_gaussian_limit():
    """Z << R: 1/r - 1/R = -Z^2 / (2 R^3) (1 - 3 Z^2 / (4 R^2) + ...), so the
    isothermal profile relative to the mid-plane cell Z_0 is
    exp(-(Z^2 - Z_0^2) / 2H^2), H = c_s / Omega, up to a relative change of
    the exponent of (3/4) (Z^2 + Z_0^2) / R^2."""
    R = 10 * AU
    cs2 = K_B * 50.0 / (MU * M_H)
    H = math.sqrt(cs2) / math.sqrt(GM / R ** 3)
    c = column(60, 50.0, R=R, Ztop=4 * H)
    rho = hse.hse_rho_gas(**c)[0]
    Z = c["Z"][0]
    r0 = math.hypot(R, Z[0])
    # the same profile relative to the mid-plane cell, then the Gaussian
    ln_got = np.log(rho / rho[0])
    ln_gauss = -(Z ** 2 - Z[0] ** 2) / (2 * H ** 2)
    bound = 0.75 * (Z ** 2 + Z[0] ** 2) / R ** 2 * np.abs(ln_gauss) * 1.05 + 1e-12
    assert np.all(np.abs(ln_got - ln_gauss) <= bound)
    assert r0 > R
