"""Pins of the oracle's mapping coefficients, right-hand side and integrator.

Mapping (Eqs. Cijk, Rijk, fragrem, Nijk), Eq. (smol) and the Bogacki-Shampine
3(2) integrator (Sec. 5) are checked against conservation laws, quadrature,
a brute-force triple sum and closed-form Smoluchowski solutions.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_2402_18471_b300 import synth


def small_disc(n_bins=12, n_cells=4, **kw):
    d = synth.make_disc(1, n_cells, n_bins, 1e-5, 1.0, 10.0, 10.0, 100.0,
                        alpha=1e-3, v_frag=100.0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def linear_disc(n_bins, m0, n_cells=1, **kw):
    d = small_disc(n_bins=n_bins, n_cells=n_cells)
    d.m, d.me = synth.linear_mass_grid(n_bins, m0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def gross_flux(o, d, rho):
    """Total mass processed per unit time, sum_k m_k n_k sum_i n_i K_ik."""
    K, pf, dv = o.kernel()
    n = rho / d.m
    return (d.m * n * np.einsum("cik,ci->ck", K, n)).sum(1)


# --------------------------------------------------------------------------
# Mapping coefficients
# --------------------------------------------------------------------------

@pytest.mark.parametrize("split", [0, 1])
def test_split_fractions_sum_to_one_and_bracket(oracle_mod, split):
    d = synth.column_1x32()
    d.split_mode = split
    o = oracle_mod.Oracle(d)
    m = d.m
    N = d.n_bins
    for i in range(N):
        for j in range(i + 1):
            oi, od = o.pair_map(i, j)
            M = m[i] + m[j]
            assert od[0] + od[1] == pytest.approx(1.0, abs=1e-15)
            if M < m[-1]:
                assert m[oi[0]] <= M < m[oi[1]] and oi[1] == oi[0] + 1
                if split == 1:
                    # number fractions conserve the number of grains
                    assert od[0] * M / m[oi[0]] + od[1] * M / m[oi[1]] == pytest.approx(1.0, rel=1e-14)
                else:
                    # mass fractions interpolate linearly in mass: the mass
                    # placed has the product's mass as its mean grain mass,
                    # which fixes the fraction given the bracketing bins
                    assert od[0] * m[oi[0]] + od[1] * m[oi[1]] == pytest.approx(M, rel=1e-14)
            # remnant + fragments carry the colliding mass (Eq. fragrem)
            assert od[4] + od[5] == pytest.approx(M, rel=1e-15)
            if od[4] > 0:
                assert od[2] + od[3] == pytest.approx(1.0, abs=1e-15)
                mr = od[4]
                if m[0] < mr < m[-1]:
                    assert m[oi[2]] <= mr < m[oi[3]] and oi[3] == oi[2] + 1
                    if split == 1:
                        assert od[2] * mr / m[oi[2]] + od[3] * mr / m[oi[3]] == pytest.approx(1.0, rel=1e-14)
                    else:
                        assert od[2] * m[oi[2]] + od[3] * m[oi[3]] == pytest.approx(mr, rel=1e-14)
            # the largest fragment min(chi m_im, m_tar) lies in bin l
            mx = min(d.chi_im * min(m[i], m[j]), max(m[i], m[j]))
            l = oi[4]
            assert d.me[l] <= mx < d.me[l + 1]


def test_equal_masses_leave_no_remnant(oracle_mod):
    """Eq. (fragrem): a collision of equal masses fragments completely (no
    remnant, 2 m_i in fragments); otherwise the remnant is less than the
    target's mass and shrinks as the projectile grows."""
    d = synth.column_1x32()
    o = oracle_mod.Oracle(d)
    m = d.m
    for i in range(d.n_bins):
        oi, od = o.pair_map(i, i)
        assert od[4] == 0.0 and od[5] == pytest.approx(2 * m[i], rel=1e-15)
        prev = None
        for j in range(i):
            oi, od = o.pair_map(i, j)
            assert 0.0 <= od[4] < m[i]
            if prev is not None:
                assert od[4] <= prev
            prev = od[4]


def test_exact_grid_hit_goes_to_one_bin(oracle_mod):
    d = linear_disc(16, 2.0 ** -30)   # power of two: sums on the grid are exact
    o = oracle_mod.Oracle(d)
    for i in range(7):
        for j in range(i + 1):
            oi, od = o.pair_map(i, j)
            assert oi[0] == i + j + 1 and od[0] == 1.0


@pytest.mark.parametrize("eta", [11.0 / 6.0, 1.5, 2.0])
def test_fragment_fractions_match_power_law_quadrature(oracle_mod, eta):
    """Eq. (Nijk) against numerical quadrature of the mass carried by the
    number distribution n(m) dm ~ m^-eta dm (Eq. fragdist) over each bin."""
    d = synth.column_1x32()
    d.eta_frag = eta
    o = oracle_mod.Oracle(d)
    tab = o.frag_table()
    me = d.me
    # mass per bin, integral of m * m^-eta dm, by quadrature in u = ln m
    parts = np.array([integrate.quad(lambda u: math.exp((2.0 - eta) * u),
                                     math.log(me[k]), math.log(me[k + 1]),
                                     epsabs=0, epsrel=1e-13)[0]
                      for k in range(d.n_bins)])
    for l in [0, 5, 23, 49]:
        tot = parts[:l + 1].sum()
        for k in range(l + 1):
            assert tab[l, k] == pytest.approx(parts[k] / tot, rel=1e-9)
        assert np.all(tab[l, l + 1:] == 0)
        assert tab[l].sum() == pytest.approx(1.0, abs=1e-14)


# --------------------------------------------------------------------------
# Right-hand side
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kmode,fmode,split", [(0, 0, 0), (0, 0, 1), (0, 1, 0), (0, 2, 0),
                                               (1, 0, 0), (2, 2, 1)])
def test_rhs_conserves_mass(oracle_mod, kmode, fmode, split):
    d = synth.column_1x32()
    d.kernel_mode, d.frag_mode, d.split_mode = kmode, fmode, split
    d.kernel_const = 1e-6 if kmode == 1 else 1e-3
    o = oracle_mod.Oracle(d)
    rho = synth.random_state(d, seed=3)
    f = o.rhs(rho)
    g = gross_flux(o, d, rho)
    assert np.all(np.abs(f.sum(1)) <= 1e-14 * g)


@pytest.mark.parametrize("fmode,split", [(0, 0), (0, 1), (2, 0), (1, 1)])
def test_rhs_two_stage_equals_bruteforce_triple_sum(oracle_mod, fmode, split):
    d = small_disc(n_bins=12, n_cells=4)
    d.frag_mode, d.split_mode = fmode, split
    o = oracle_mod.Oracle(d)
    rho = synth.random_state(d, seed=7, spread=3)
    f = o.rhs(rho)
    fb = o.rhs_bruteforce(rho)
    g = gross_flux(o, d, rho)
    assert np.all(np.abs(f - fb).max(1) <= 1e-14 * g)


def test_rhs_number_rate_constant_kernel(oracle_mod):
    """Constant kernel, no fragmentation, number-conserving split: the total
    number obeys dN/dt = -K N^2 / 2 exactly (while products stay on the grid)."""
    d = synth.column_1x32()
    d.kernel_mode, d.kernel_const, d.frag_mode, d.split_mode = 1, 3e-7, 1, 1
    o = oracle_mod.Oracle(d)
    rho = synth.random_state(d, seed=4, spread=3)
    rho[:, 40:] = 0.0   # keep every product below the top bin
    f = o.rhs(rho)
    n = rho / d.m
    Nn = n.sum(1)
    assert np.allclose((f / d.m).sum(1), -0.5 * d.kernel_const * Nn ** 2, rtol=1e-12)


def test_rhs_single_species_fragmentation(oracle_mod):
    """Equal-mass collisions that always fragment leave no remnant: every
    gram removed from bin i reappears in bins k <= i."""
    d = synth.column_1x32()
    d.frag_mode = 2
    o = oracle_mod.Oracle(d)
    rho = np.zeros((d.n_cells, d.n_bins))
    rho[:, 30] = 1e-14
    f = o.rhs(rho)
    assert np.all(f[:, 31:] == 0)
    assert np.all(f[:, :30] > 0)
    assert np.allclose(f[:, :31].sum(1), 0, atol=1e-14 * np.abs(f[:, 30]).max())


# --------------------------------------------------------------------------
# Integrator and closed-form solutions
# --------------------------------------------------------------------------

def test_bs3_one_step_linear_stability_polynomial(oracle_mod):
    """One BS3 step of y' = lam y is exactly 1 + z + z^2/2 + z^3/6."""
    for z in [-0.3, -1.7, 0.2, -2.4]:
        out = oracle_mod.bs3_scalar(z, 1.0, 1.0, 1.0, fixed_steps=1)
        assert out[0] == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6, rel=1e-15)


def test_bs3_third_order_convergence(oracle_mod):
    errs = []
    for n in [20, 40, 80]:
        out = oracle_mod.bs3_scalar(-1.3, 1.0, 2.0, 2.0 / n, fixed_steps=n)
        errs.append(abs(out[0] - math.exp(-2.6)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.0 and 7.0 < r2 < 9.0


def test_bs3_adaptive_error_tracks_tolerance(oracle_mod):
    exact = math.exp(-5.0)
    prev_n = 0
    for rtol in [1e-3, 1e-5, 1e-7]:
        out = oracle_mod.bs3_scalar(-1.0, 1.0, 5.0, 0.0, rtol=rtol, atol=1e-14)
        assert abs(out[0] - exact) / exact < 50 * rtol
        assert out[1] > prev_n
        prev_n = out[1]


def _bs3_controller_closed_form(lam, y0, T, h, rtol, atol):
    """The step controller's reading (per-cell max-norm error against atol +
    rtol max(|y|, |y'|); accept when E <= 1 and y' >= -atol; next step h E
    -> h min(5, max(0.2, 0.9 E^-1/3)), 5 at E = 0; a rejected step shrinks
    by max(0.2, 0.9 E^-1/3); the last step cut to the end keeps h; h0 = 0.1
    (|y| + atol) / |f|) on y' = lam y, with the local error taken from the
    published embedded weights (7/24, 1/4, 1/3, 1/8) and the stage
    polynomials of a linear problem: k2 = lam y (1 + z/2), k3 = lam y (1 +
    3z/4 + 3z^2/8), y' = y R(z), R = 1 + z + z^2/2 + z^3/6, z = lam h."""
    t, y, nacc, nrej = 0.0, y0, 0, 0
    if not h > 0.0:
        h = min(0.1 * (abs(y) + atol) / abs(lam * y), T)
    while t < T:
        last = h >= T - t
        hs = T - t if last else h
        z = lam * hs
        R = 1 + z + z * z / 2 + z ** 3 / 6
        Rhat = 1 + z * (7 / 24 + (1 + z / 2) / 4 + (1 + 3 * z / 4 + 3 * z * z / 8) / 3 + R / 8)
        y1 = y * R
        E = abs(y * (R - Rhat)) / (atol + rtol * max(abs(y), abs(y1)))
        if E <= 1.0 and y1 >= -atol:
            t = T if last else t + hs
            y = y1
            nacc += 1
            fac = min(5.0, max(0.2, 0.9 * E ** (-1 / 3))) if E > 0 else 5.0
            if not (last and hs < h):
                h = hs * fac
        else:
            nrej += 1
            h = hs * max(0.2, 0.9 * E ** (-1 / 3))
    return y, nacc, nrej


@pytest.mark.parametrize("lam,y0,T,h0,rtol", [
    (-1.0, 1.0, 5.0, 0.0, 1e-3),      # automatic first step, smooth decay
    (-1.0, 1.0, 5.0, 0.0, 1e-6),
    (-10.0, 2.0, 3.0, 2.0, 1e-4),     # a first step far too long: rejections at the 0.2 clamp
    (0.7, 1.0, 4.0, 1e-6, 1e-5),      # growth from a tiny step: the factor-5 clamp
    (-3.0, 1.0, 2.0, 0.05, 1e-2),     # the paper's rtol
])
def test_bs3_step_controller_matches_its_closed_form(oracle_mod, lam, y0, T, h0, rtol):
    """Pins the controller constants and rules (not given by the paper) and
    the embedded error estimate: the oracle's accepted and rejected step
    counts and end state on y' = lam y equal those of the rules applied to
    the closed-form stage values."""
    y, nacc, nrej = _bs3_controller_closed_form(lam, y0, T, h0, rtol, 1e-12)
    out = oracle_mod.bs3_scalar(lam, y0, T, h0, rtol=rtol, atol=1e-12)
    assert (int(out[1]), int(out[2])) == (nacc, nrej)
    assert out[0] == pytest.approx(y, rel=1e-12)
    if h0 == 2.0:
        assert nrej >= 2


def _constant_kernel_analytic(N, N0, tau):
    k = np.arange(1, N + 1)
    return N0 * (tau / 2) ** (k - 1) / (1 + tau / 2) ** (k + 1)


@pytest.mark.parametrize("split", [0, 1])
def test_constant_kernel_matches_closed_form(oracle_mod, split):
    """Constant kernel on the linear grid m_k = (k+1) m0 from a monodisperse
    start: n_k(t) = N0 (tau/2)^(k-1) / (1 + tau/2)^(k+1), tau = K N0 t
    (the analytic test of Sec. 5.1)."""
    N, m0, N0, K = 64, 2.0 ** -40, 1.0, 1e-6
    d = linear_disc(N, m0, kernel_mode=1, kernel_const=K, frag_mode=1,
                    split_mode=split, rtol=1e-8, atol_rel=1e-25)
    rho = np.zeros((1, N)); rho[0, 0] = N0 * m0
    tau = 1.0
    res = oracle_mod.Oracle(d).step(rho, tau / (K * N0))
    assert res["status"][0] == 0
    n = res["rho"][0] / d.m
    ref = _constant_kernel_analytic(N, N0, tau)
    sel = ref > 1e-12 * N0
    assert np.allclose(n[sel], ref[sel], rtol=2e-5)
    assert res["rho"].sum() == pytest.approx(rho.sum(), rel=1e-13)


def test_additive_kernel_matches_golovin(oracle_mod):
    """Additive kernel K = beta (m_i + m_j) from a monodisperse start:
    n_k = N0 (1-g) (k g)^(k-1) exp(-k g) / k!, g = 1 - exp(-beta N0 m0 t)."""
    N, m0, N0 = 96, 2.0 ** -40, 1.0
    beta = 1e-6 / m0
    d = linear_disc(N, m0, kernel_mode=2, kernel_const=beta, frag_mode=1,
                    split_mode=0, rtol=1e-8, atol_rel=1e-25)
    rho = np.zeros((1, N)); rho[0, 0] = N0 * m0
    g = 0.4
    t = -math.log(1 - g) / (beta * N0 * m0)
    res = oracle_mod.Oracle(d).step(rho, t)
    assert res["status"][0] == 0
    n = res["rho"][0] / d.m
    k = np.arange(1, N + 1)
    ref = np.exp(np.log(N0 * (1 - g)) + (k - 1) * np.log(k * g) - k * g - special.gammaln(k + 1))
    sel = ref > 1e-10 * N0
    assert np.allclose(n[sel], ref[sel], rtol=3e-5)
    assert n.sum() == pytest.approx(N0 * (1 - g), rel=1e-6)


def log_disc(per_decade, m0, lo=-3, hi=4, **kw):
    """One cell on a logarithmic mass grid of per_decade bins per decade from
    10^lo m0 to 10^hi m0, edges at the geometric midpoints of the centres."""
    N = per_decade * (hi - lo)
    r = 10.0 ** (1.0 / per_decade)
    m = m0 * 10.0 ** lo * r ** (np.arange(N) + 0.5)
    me = np.empty(N + 1)
    me[1:-1] = np.sqrt(m[1:] * m[:-1])
    me[0], me[-1] = m[0] / math.sqrt(r), m[-1] * math.sqrt(r)
    d = small_disc(n_bins=N, n_cells=1)
    d.m, d.me = m, me
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def _exp_bin_mass(me, m0, s=1.0, N0=1.0):
    """Mass per bin of n(m) = N0 / (m0 s^2) exp(-m / (m0 s)): the integral of
    m n(m) over each bin, N0 m0 [(1 + a) e^-a]_b^a with a = m / (m0 s)."""
    a, b = me[:-1] / (m0 * s), me[1:] / (m0 * s)
    return N0 * m0 * ((1 + a) * np.exp(-a) - (1 + b) * np.exp(-b))


@pytest.mark.parametrize("kind", ["constant", "additive"])
@pytest.mark.parametrize("split", [0, 1])
def test_log_grid_converges_to_continuous_solutions(oracle_mod, kind, split):
    """On logarithmic grids (the method's own) from an exponential start,
    n(m, 0) = N0/m0 exp(-m/m0), the binned solution approaches the continuous
    one: constant kernel n = N0 / (m0 s^2) exp(-m / (m0 s)), s = 1 + tau/2,
    tau = K N0 t; additive kernel (Golovin) m n = N0 (1-g)/sqrt(g) exp(-(1+g)x)
    I1(2 x sqrt(g)), x = m/m0, g = 1 - exp(-beta N0 m0 t).  The L1 error of
    the mass distribution must fall by more than 3 for each doubling of the
    bins per decade (second order) and be below 1 % at 20 bins per decade."""
    m0 = 2.0 ** -40
    errs = []
    for per_decade in (5, 10, 20):
        if kind == "constant":
            K, tau = 1e-6, 2.0
            d = log_disc(per_decade, m0, kernel_mode=1, kernel_const=K, frag_mode=1, split_mode=split,
                         rtol=1e-8, atol_rel=1e-25)
            t = tau / K
            want = _exp_bin_mass(d.me, m0, s=1 + tau / 2)
        else:
            beta, g = 1e-6 / m0, 0.5
            d = log_disc(per_decade, m0, kernel_mode=2, kernel_const=beta, frag_mode=1, split_mode=split,
                         rtol=1e-8, atol_rel=1e-25)
            t = -math.log(1 - g) / (beta * m0)
            sg = math.sqrt(g)
            f = lambda x: (1 - g) / sg * special.i1e(2 * x * sg) * math.exp(-x * (1 - sg) ** 2)
            want = np.array([m0 * integrate.quad(f, d.me[k] / m0, d.me[k + 1] / m0, epsrel=1e-12, limit=200)[0]
                             for k in range(d.n_bins)])
        rho = _exp_bin_mass(d.me, m0)[None]
        res = oracle_mod.Oracle(d).step(rho, t)
        assert res["status"][0] == 0
        assert res["rho"].sum() == pytest.approx(rho.sum(), rel=1e-12)
        errs.append(np.abs(res["rho"][0] - want).sum() / want.sum())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
    assert errs[2] < 1e-2, errs


def test_fixed_step_convergence_on_constant_kernel(oracle_mod):
    """Third-order convergence of the coagulation integration itself."""
    N, m0, N0, K = 48, 2.0 ** -40, 1.0, 1e-6
    d = linear_disc(N, m0, kernel_mode=1, kernel_const=K, frag_mode=1)
    o = oracle_mod.Oracle(d)
    rho = np.zeros((1, N)); rho[0, 0] = N0 * m0
    T = 1.0 / (K * N0)
    ref = _constant_kernel_analytic(N, N0, 1.0) * d.m
    errs = []
    for ns in [8, 16, 32]:
        hs = np.full((1, ns), T / ns)
        y = o.replay(rho, hs, np.array([ns]))
        errs.append(np.abs(y[0, :10] - ref[:10]).max())
    assert 6.5 < errs[0] / errs[1] < 9.5 and 6.5 < errs[1] / errs[2] < 9.5


def test_physical_step_conserves_mass_and_replay_is_exact(oracle_mod):
    d = synth.column_1x32()
    o = oracle_mod.Oracle(d)
    res = o.step(d.rho0, d.t_span, log_cap=5000)
    assert np.all(res["status"] == 0)
    assert np.allclose(res["rho"].sum(1), d.rho0.sum(1), rtol=1e-13)
    # the same accepted step sequence replayed gives the same state
    y = o.replay(d.rho0, res["log"], res["n_log"])
    assert np.array_equal(y, res["rho"])
    # growth happened: mass moved above the initial 1 um cut
    a = d.extra["a"]
    assert (res["rho"][:, a > 2e-4].sum(1) > 0.01 * d.rho0.sum(1)).any()


def test_step_limits_report_status(oracle_mod):
    d = synth.column_1x32().subset([0, 1])
    d.max_substeps = 5
    res = oracle_mod.Oracle(d).step(d.rho0, d.t_span)
    assert np.all(res["status"] == 4)
    assert np.all(res["n_acc"] + res["n_rej"] == 5)


def test_empty_cell_passes_through(oracle_mod):
    """A cell without dust has atol = 0 and a zero right-hand side: its error
    ratio is 0 (not 0/0), so it takes one step of t_span and stays empty,
    while the cell next to it integrates as it would alone."""
    d = synth.column_1x32().subset([0, 1])
    rho0 = d.rho0.copy()
    rho0[1] = 0.0
    o = oracle_mod.Oracle(d)
    res = o.step(rho0, d.t_span)
    assert np.all(res["status"] == 0)
    assert res["n_acc"][1] == 1 and res["n_rej"][1] == 0
    assert np.all(res["rho"][1] == 0.0)
    alone = oracle_mod.Oracle(d.subset([0])).step(rho0[:1], d.t_span)
    assert np.array_equal(res["rho"][0], alone["rho"][0])
