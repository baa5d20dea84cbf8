"""Pins of the oracle's discrete adjoint (gradients of L = sum w rho(T) after a
fixed BS3 step sequence) against central finite differences of the oracle's
own replay, for the initial densities, the per-cell alpha and v_frag."""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth


def adj_disc():
    # A small column over 0.1-10 um (mass ratio 1e6) with strong
    # fragmentation (v_frag 1 cm/s) so that the p_frag and turbulence
    # derivatives carry weight.  Wider size ranges are avoided here: the
    # literal FP64 right-hand side adds and removes m_i-sized masses for
    # sweep-up pairs, leaving rounding noise of ~1e-16 m_max/m_min of the
    # transfer, which finite differences would pick up.
    d = synth.make_disc(1, 4, 14, 1e-5, 1e-3, 10.0, 10.0, 3000.0, alpha=2e-3, v_frag=1.0, seed=3)
    d.rho0 = synth.random_state(d, seed=8, spread=2)
    return d


def loss_and_steps(oracle_mod, d, w, hs=None, n_h=None):
    o = oracle_mod.Oracle(d)
    if hs is None:
        ref = o.step(d.rho0, d.t_span, log_cap=4000)
        hs, n_h = ref["log"], ref["n_log"]
    y = o.replay(d.rho0, hs, n_h)
    return float((w * y).sum()), hs, n_h


def test_adjoint_matches_finite_differences(oracle_mod):
    d = adj_disc()
    rng = np.random.default_rng(2)
    w = rng.standard_normal((d.n_cells, d.n_bins)) / d.rho0.sum(1, keepdims=True)
    L0, hs, n_h = loss_and_steps(oracle_mod, d, w)
    g_rho0, g_alpha, g_vf = oracle_mod.Oracle(d).vjp(d.rho0, hs, n_h, w)

    def L_of(mod):
        dd = adj_disc()
        mod(dd)
        return loss_and_steps(oracle_mod, dd, w, hs, n_h)[0]

    # initial densities, every component, relative step 1e-5 (truncation
    # ~1e-10, rounding ~1e-7 of the largest component)
    o = oracle_mod.Oracle(d)
    floor = 1e-6 * abs(g_rho0).max()
    for c in range(d.n_cells):
        for k in range(d.n_bins):
            e = 1e-5 * max(d.rho0[c, k], 1e-3 * d.rho0[c].sum())
            rp, rm = d.rho0.copy(), d.rho0.copy()
            rp[c, k] += e
            rm[c, k] -= e
            fd = (float((w * o.replay(rp, hs, n_h)).sum())
                  - float((w * o.replay(rm, hs, n_h)).sum())) / (2 * e)
            assert g_rho0[c, k] == pytest.approx(fd, rel=2e-6, abs=floor)
    # per-cell alpha.  A central difference with step e = 1e-5 alpha has
    # truncation ~1e-10 and rounding ~1e-16 |L-terms| / e ~ 1e-7 of the
    # largest gradient, so small components get an absolute floor of 1e-6 of
    # the largest one.
    for c in range(d.n_cells):
        e = 1e-5 * d.alpha[c]
        fd = (L_of(lambda dd: dd.alpha.__setitem__(c, dd.alpha[c] + e))
              - L_of(lambda dd: dd.alpha.__setitem__(c, dd.alpha[c] - e))) / (2 * e)
        assert g_alpha[c] == pytest.approx(fd, rel=1e-5, abs=1e-6 * abs(g_alpha).max())
    # v_frag
    e = 1e-5 * d.v_frag
    fd = (L_of(lambda dd: setattr(dd, "v_frag", dd.v_frag + e))
          - L_of(lambda dd: setattr(dd, "v_frag", dd.v_frag - e))) / (2 * e)
    assert g_vf == pytest.approx(fd, rel=1e-6)


def test_adjoint_dot_product_identity(oracle_mod):
    """<J u, w> = <u, J^T w> for the linearised map rho0 -> rho(T), with J u
    taken by a central difference along a random direction u."""
    d = adj_disc()
    rng = np.random.default_rng(5)
    w = rng.standard_normal((d.n_cells, d.n_bins))
    u = rng.standard_normal((d.n_cells, d.n_bins)) * d.rho0
    o = oracle_mod.Oracle(d)
    ref = o.step(d.rho0, d.t_span, log_cap=4000)
    hs, n_h = ref["log"], ref["n_log"]
    g_rho0, _, _ = o.vjp(d.rho0, hs, n_h, w)
    # eps = 1e-5: truncation ~1e-10, rounding ~1e-11 relative
    eps = 1e-5
    Jp = o.replay(d.rho0 + eps * u, hs, n_h)
    Jm = o.replay(d.rho0 - eps * u, hs, n_h)
    lhs = ((Jp - Jm) / (2 * eps) * w).sum()
    rhs = (u * g_rho0).sum()
    assert lhs == pytest.approx(rhs, rel=1e-8)


def test_adjoint_of_zero_steps_is_identity(oracle_mod):
    d = adj_disc()
    w = np.random.default_rng(1).standard_normal((d.n_cells, d.n_bins))
    g, ga, gv = oracle_mod.Oracle(d).vjp(d.rho0, np.zeros((d.n_cells, 1)),
                                         np.zeros(d.n_cells, dtype=np.int64), w)
    assert np.array_equal(g, w) and np.all(ga == 0) and gv == 0
