"""Pins of the oracle's per-cell spans and of the sub-cycling trigger (Sec. 6).

The coagulation solver sub-cycles: it takes its own steps inside the global
steps of the disc model, and a cell is brought up to date once one (by
default) of its last sub-steps has elapsed in global time.  These tests pin
the oracle's version of that against facts that do not depend on it:
independence of cells, conservation of integrated time, the trigger's
invariant, and the closed-form constant-kernel solution reached through
many sub-cycled updates (the evolution composes over time, Sec. 5.1).
"""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

from test_oracle_rhs import _constant_kernel_analytic, linear_disc


def test_spans_skip_cells_and_match_single_cell_steps(oracle_mod):
    """Per-cell spans: cells with span <= 0 are untouched bitwise; every
    other cell ends exactly as a step of its own span taken alone."""
    d = synth.column_1x32().subset(list(range(6)))
    o = oracle_mod.Oracle(d)
    T = d.t_span
    spans = np.array([T, 0.0, 0.25 * T, -1.0, 3.0 * T, np.nan])
    dt0 = np.array([0.0, 5.0, 0.0, 7.0, 0.0, 9.0])
    res = o.step(d.rho0, spans, dt0, log_cap=4000)
    assert np.all(res["status"] == 0)
    for c in (1, 3, 5):
        assert np.array_equal(res["rho"][c], d.rho0[c])
        assert res["dt"][c] == dt0[c] and res["n_acc"][c] == 0 and res["n_log"][c] == 0
    for c in (0, 2, 4):
        alone = oracle_mod.Oracle(d.subset([c])).step(d.rho0[c:c + 1], spans[c], log_cap=4000)
        assert np.array_equal(res["rho"][c], alone["rho"][0])
        assert res["n_acc"][c] == alone["n_acc"][0]
        # the accepted steps add up to the cell's span
        assert res["log"][c, :res["n_log"][c]].sum() == pytest.approx(spans[c], rel=1e-13)


def test_subcycle_accounts_for_all_global_time(oracle_mod):
    """Over many global steps every cell's integrated time plus its pending
    time is the global time elapsed, and a cell left pending has not yet
    reached trigger x its last sub-step."""
    d = synth.column_1x32().subset([0, 5, 11, 17, 23, 31])
    o = oracle_mod.Oracle(d)
    n = d.n_cells
    y, dt, pend = d.rho0.copy(), np.zeros(n), np.zeros(n)
    done = np.zeros(n)
    n_upd = np.zeros(n, dtype=int)
    M, dtg = 40, d.t_span / 40
    for _ in range(M):
        res = o.subcycle(y, pend, dt, dtg, log_cap=4000)
        assert np.all(res["status"] == 0)
        due = res["spans"] > 0
        # pending cells: under one sub-step; updated cells: restarted
        assert np.all(res["pending"][~due] < dt[~due])
        assert np.all(res["pending"][due] == 0.0)
        for c in np.flatnonzero(due):
            done[c] += res["log"][c, :res["n_log"][c]].sum()
        n_upd += due
        y, dt, pend = res["rho"], res["dt"], res["pending"]
    assert np.allclose(done + pend, M * dtg, rtol=1e-12)
    # the first call updates every cell (no sub-step yet); afterwards cells
    # whose sub-steps outgrow the global step are updated less often
    assert np.all(n_upd >= 1) and n_upd.min() < M
    assert np.allclose(y.sum(1), d.rho0.sum(1), rtol=1e-12)


def test_subcycle_trigger_zero_like_updates_every_step(oracle_mod):
    """A trigger far below one updates every cell at every global step: the
    same as stepping each global step with the last sub-step carried."""
    d = synth.column_1x32().subset([2, 9])
    o = oracle_mod.Oracle(d)
    dtg = d.t_span / 8
    y1, dt1, pend = d.rho0.copy(), np.zeros(2), np.zeros(2)
    y2, dt2 = d.rho0.copy(), np.zeros(2)
    for _ in range(8):
        r1 = o.subcycle(y1, pend, dt1, dtg, trigger=1e-300)
        assert np.all(r1["spans"] == dtg)
        y1, dt1, pend = r1["rho"], r1["dt"], r1["pending"]
        r2 = o.step(y2, dtg, dt2)
        y2, dt2 = r2["rho"], r2["dt"]
    assert np.array_equal(y1, y2) and np.array_equal(dt1, dt2)


def test_subcycled_constant_kernel_matches_closed_form(oracle_mod):
    """Constant kernel from a monodisperse start (Sec. 5.1), advanced by
    many global steps much shorter than the coagulation sub-steps, then
    brought up to date at tau = K N0 t = 1: the closed form at tau = 1."""
    N, m0, N0, K = 64, 2.0 ** -40, 1.0, 1e-6
    d = linear_disc(N, m0, kernel_mode=1, kernel_const=K, frag_mode=1,
                    split_mode=0, rtol=1e-6, atol_rel=1e-25)
    o = oracle_mod.Oracle(d)
    rho = np.zeros((1, N)); rho[0, 0] = N0 * m0
    T = 1.0 / (K * N0)
    M = 2000
    dt, pend, n_upd = np.zeros(1), np.zeros(1), 0
    for _ in range(M):
        res = o.subcycle(rho, pend, dt, T / M)
        n_upd += int(res["spans"][0] > 0)
        rho, dt, pend = res["rho"], res["dt"], res["pending"]
    if pend[0] > 0:                              # bring the cell up to date
        rho = o.step(rho, pend, dt)["rho"]
    assert 1 < n_upd < M
    n = rho[0] / d.m
    ref = _constant_kernel_analytic(N, N0, 1.0)
    sel = ref > 1e-12 * N0
    assert np.allclose(n[sel], ref[sel], rtol=1e-5)
