"""Pins of the oracle's per-pair physics against facts independent of its code.

Relative velocities (Sec. 5, Eqs. vbrown and OCVrel), the fragmentation
probability (Eq. p_frag), the Epstein stopping time (Eq. t_stop) and the mass
grid of Sec. 7.
"""
import json
import os

import numpy as np
import pytest
from scipy import stats

from paper_2402_18471_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _one_cell(**kw):
    d = synth.column_1x32()
    d = d.subset([0])
    for k, v in kw.items():
        arr = getattr(d, k)
        if isinstance(arr, np.ndarray):
            arr[...] = v
        else:
            setattr(d, k, v)
    return d


def test_mass_grid_ratio_matches_paper():
    """Sec. 7: 100 bins (0.1 um-0.5 cm) and 135 bins (0.1 um-20 cm) give 1.38."""
    g = json.load(open(GOLD))["mass_ratio_grids"]
    for case in g["cases"]:
        m, me, a = synth.log_mass_grid(case["n_bins"], case["a_min_cm"], case["a_max_cm"], 1.6)
        r = m[1:] / m[:-1]
        assert np.allclose(r, r[0], rtol=1e-12)
        assert round(r[0], g["printed_digits"]) == case["ratio"]
        assert np.all(me[:-1] < m) and np.all(m < me[1:])


def test_grain_size_from_mass(oracle_mod):
    d = synth.column_1x32()
    ph = oracle_mod.Oracle(d).cell_physics(0)
    assert np.allclose(ph["a"], d.extra["a"], rtol=1e-13)


def test_vrel_tiny_particle_limit(oracle_mod):
    """OC07 tiny-particle limit: V_rel^2 -> Re^1/2 (St1 - St2)^2 for St << Re^-1/2."""
    Re = 1e8
    d = Re ** -0.5
    for s1, s2 in [(1e-7, 1e-8), (3e-7, 2.9e-7), (5e-8, 1e-9)]:
        v = oracle_mod.vrel2(s1, s2, Re)
        ref = Re ** 0.5 * (s1 - s2) ** 2
        assert v == pytest.approx(ref, rel=2e-2 + 5 * s1 / d)


@pytest.mark.parametrize("eps", [0.01, 0.1, 0.3, 0.7, 1.0])
def test_vrel_intermediate_regime_beta(oracle_mod, eps):
    """OC07 Eq. 28: V_rel^2 = beta St1 with
    beta = 2y - (1+eps) + 2/(1+eps) (1/(1+y) + eps^3/(y+eps)), y = 1.6,
    for Re^-1/2 << St2 = eps St1 << 1."""
    y = 1.6
    beta = 2 * y - (1 + eps) + 2 / (1 + eps) * (1 / (1 + y) + eps ** 3 / (y + eps))
    St1 = 1e-5
    v = oracle_mod.vrel2(St1, eps * St1, 1e22)
    assert v / St1 == pytest.approx(beta, rel=2e-3)


def test_vrel_heavy_limit(oracle_mod):
    """OC07 heavy-particle limit: V_rel^2 -> 1/(1+St1) + 1/(1+St2) for St >> 1."""
    for s1, s2 in [(1e3, 2e2), (5e4, 5e4), (1e5, 3e3)]:
        v = oracle_mod.vrel2(s1, s2, 1e10)
        ref = 1 / (1 + s1) + 1 / (1 + s2)
        assert v == pytest.approx(ref, rel=5e-2)


def test_vrel_symmetric_and_continuous(oracle_mod):
    for s in [1e-4, 1e-2, 0.3, 2.0]:
        assert oracle_mod.vrel2(s, 0.5 * s, 1e9) == oracle_mod.vrel2(0.5 * s, s, 1e9)
    # equal Stokes numbers: only the class II response survives, which stays
    # positive and continuous across the St* = 1 clamp
    vals = [oracle_mod.vrel2(s, s, 1e9) for s in np.linspace(0.5, 0.8, 31)]
    assert min(vals) > 0 and np.max(np.abs(np.diff(vals))) < 0.05


def test_brownian_velocity_is_maxwellian_mean_relative_speed(oracle_mod):
    """v_BM (Eq. vbrown) equals the mean |v1 - v2| of two Maxwellian grains:
    Monte Carlo with each velocity component ~ N(0, k_B T / m)."""
    # alpha -> 0 gives Re << 1: the clamp makes v_turb exactly zero; eta = 0
    # and Z = 0 switch off the laminar terms, so dv = v_BM.
    d = _one_cell(alpha=1e-30, eta=0.0, Z=0.0)
    o = oracle_mod.Oracle(d)
    K, pf, dv = o.kernel()
    rng = np.random.default_rng(5)
    kT = synth.CONST["k_B"] * d.T[0]
    for i, j in [(0, 0), (3, 0), (10, 4)]:
        n = 400_000
        v1 = rng.standard_normal((n, 3)) * np.sqrt(kT / d.m[i])
        v2 = rng.standard_normal((n, 3)) * np.sqrt(kT / d.m[j])
        mc = np.linalg.norm(v1 - v2, axis=1).mean()
        assert dv[0, i, j] == pytest.approx(mc, rel=5e-3)


def test_pfrag_is_gamma_survival(oracle_mod):
    """Eq. (p_frag) is the probability that the squared speed exceeds v_f^2
    when it follows a Gamma(shape 2, scale 2 dv^2 / 3) law (Maxwellian
    fragmentation model); limits 0 and 1 and monotone decrease with v_f."""
    for dv in [10.0, 100.0, 350.0, 3000.0]:
        for vf in [30.0, 100.0, 1000.0]:
            ref = stats.gamma(a=2.0, scale=2.0 * dv * dv / 3.0).sf(vf * vf)
            assert oracle_mod.pfrag(dv, vf) == pytest.approx(ref, rel=1e-12, abs=1e-300)
    assert oracle_mod.pfrag(1e-3, 100.0) == 0.0
    assert oracle_mod.pfrag(1e9, 100.0) == pytest.approx(1.0, abs=1e-12)
    p = [oracle_mod.pfrag(100.0, vf) for vf in np.linspace(1, 500, 200)]
    assert np.all(np.diff(p) < 0)


def test_epstein_stokes_number(oracle_mod):
    """Eq. (t_stop): St = rho_m a Omega / (rho_g v_th) with v_th the mean
    molecular speed of the gas; checked against a Monte Carlo mean speed."""
    d = synth.column_1x32()
    o = oracle_mod.Oracle(d)
    c = 5
    ph = o.cell_physics(c)
    kT = synth.CONST["k_B"] * d.T[c]
    mgas = d.mu * synth.CONST["m_H"]
    rng = np.random.default_rng(1)
    vth_mc = np.linalg.norm(rng.standard_normal((600_000, 3)) * np.sqrt(kT / mgas), axis=1).mean()
    Om = np.sqrt(synth.CONST["G"] * d.Mstar / (d.R[c] ** 2 + d.Z[c] ** 2) ** 1.5)
    St_mc = d.rho_m * ph["a"] * Om / (d.rho_gas[c] * vth_mc)
    assert np.allclose(ph["St"], St_mc, rtol=5e-3)
    assert ph["cs"] ** 2 == pytest.approx(kT / mgas, rel=1e-12)


def test_kernel_symmetry_and_geometry(oracle_mod):
    d = synth.column_1x32()
    o = oracle_mod.Oracle(d)
    K, pf, dv = o.kernel()
    assert np.allclose(K, np.swapaxes(K, 1, 2), rtol=1e-14)
    # exp(-x) with x up to ~500 amplifies last-ulp differences of dv
    assert np.allclose(pf, np.swapaxes(pf, 1, 2), rtol=1e-11, atol=1e-300)
    a = d.extra["a"]
    sig = np.pi * (a[:, None] + a[None, :]) ** 2
    assert np.allclose(K / dv, sig[None], rtol=1e-12)
    assert np.all((pf >= 0) & (pf <= 1))


def test_turbulent_term_scales_with_alpha(oracle_mod):
    """v_turb^2 = alpha c_s^2 V_rel^2 (Sec. 5): with Brownian and laminar
    parts removed by differencing, dv^2 grows linearly in alpha times the
    ratio of V_rel^2 (which moves with Re, itself linear in alpha)."""
    o1 = oracle_mod.Oracle(_one_cell(eta=0.0, Z=0.0))
    d2 = _one_cell(eta=0.0, Z=0.0)
    d2.alpha[:] = 4e-3
    o2 = oracle_mod.Oracle(d2)
    o0 = oracle_mod.Oracle(_one_cell(alpha=1e-30, eta=0.0, Z=0.0))
    dv1 = o1.kernel()[2][0]; dv2 = o2.kernel()[2][0]; dv0 = o0.kernel()[2][0]
    t1 = dv1 ** 2 - dv0 ** 2
    t2 = dv2 ** 2 - dv0 ** 2
    ph1 = o1.cell_physics(0); ph2 = o2.cell_physics(0)
    assert ph2["Re"] == pytest.approx(4.0 * ph1["Re"], rel=1e-12)
    N = d2.n_bins
    v1 = np.array([[oracle_mod.vrel2(ph1["St"][i], ph1["St"][j], ph1["Re"]) for j in range(N)] for i in range(N)])
    v2 = np.array([[oracle_mod.vrel2(ph2["St"][i], ph2["St"][j], ph2["Re"]) for j in range(N)] for i in range(N)])
    big = t1 > 1e-6 * dv1 ** 2
    assert np.allclose((t2 / t1)[big], (4.0 * v2 / v1)[big], rtol=1e-8)
