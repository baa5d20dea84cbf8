"""GPU parity of per-cell integration spans and of sub-cycled coagulation
(Sec. 6) against the FP64 CPU oracle, through the C ABI.

The coagulation solver takes its own sub-steps inside the global steps of
the disc model; a cell is brought up to date once one of its last sub-steps
has elapsed in global time.  Both sides take that decision in FP64 from the
same pending time and last sub-step, so the set of updated cells and the
pending times must agree exactly.  The integrations themselves are held to
the tolerances of the whole-grid step: 1e-10 relative for the FP64 path (the
same accepted steps as the oracle), and for the mixed path the oracle's
replay of the GPU's own accepted steps within 1e-5 |rho| + 1e-10 S.
"""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def check_mixed(out, want, S):
    r = np.abs(out - want) / (1e-5 * np.abs(want) + 1e-10 * S[:, None])
    assert r.max() <= 1.0, f"error {r.max():.3f} x (1e-5 |rho| + 1e-10 S)"


def check_fp64(out, want, S):
    assert np.all(np.abs(out - want) <= 1e-10 * np.abs(want) + 1e-20 * S[:, None])


def log_sums(logs, n):
    """Sum of each cell's first n[c] logged steps (later entries are left
    from earlier calls)."""
    return np.where(np.arange(logs.shape[1])[None, :] < n[:, None], logs, 0.0).sum(1)


def mixed_spans(d, seed):
    """Spans of 0.1 to 2 t_span, with about a third of the cells skipped
    (span 0 or negative)."""
    rng = np.random.default_rng(seed)
    s = d.t_span * rng.choice([0.0, -1.0, 0.1, 0.5, 1.0, 2.0], size=d.n_cells)
    s[0] = d.t_span
    return s


CASES = {
    "column_1x32_N50": lambda: synth.column_1x32(),
    "N40_4736_cells": lambda: synth.make_disc(74, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_step_spans_matches_oracle(coag_mod, oracle_mod, precision, case):
    d = CASES[case]()
    if precision == "fp64" and d.n_cells > 64:
        d = d.subset(np.arange(0, d.n_cells, d.n_cells // 48)[:48])
    spans = mixed_spans(d, seed=3)
    act = spans > 0
    dt0 = np.where(act, 0.0, 42.0)                # skipped cells keep their dt
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(4000)
    y = g.state(d.rho0)
    dt = torch.as_tensor(dt0, device="cuda")
    st = g.step_spans(y, torch.as_tensor(spans, device="cuda"), dt)
    assert st["status"] == 0 and st["n_failed"] == 0
    out, dto = y.cpu().numpy(), dt.cpu().numpy()
    n, logs = rec["n"].cpu().numpy(), rec["dt"].cpu().numpy()
    assert st["accepted"] == n.sum()
    assert np.array_equal(out[~act], d.rho0[~act]) and np.all(dto[~act] == 42.0) and np.all(n[~act] == 0)
    assert np.all(n[act] >= 1)
    assert np.allclose(log_sums(logs, n)[act], spans[act], rtol=1e-12)
    S = d.rho0.sum(1)
    if precision == "fp64":
        ref = oracle_mod.Oracle(d).step(d.rho0, spans, dt0, log_cap=4000)
        assert np.array_equal(n, ref["n_log"])
        assert np.allclose(logs, ref["log"], rtol=1e-9, atol=0)
        check_fp64(out, ref["rho"], S)
        assert np.allclose(dto, ref["dt"], rtol=1e-9)
    else:
        cells = np.flatnonzero(act)
        cells = cells[np.unique(np.linspace(0, cells.size - 1, min(16, cells.size)).astype(int))]
        want = oracle_mod.Oracle(d.subset(cells)).replay(d.rho0[cells], logs[cells], n[cells])
        check_mixed(out[cells], want, S[cells])
        assert st["mass_err_max"] < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subcycle_matches_oracle(coag_mod, oracle_mod, precision):
    """Twelve global steps of t_span / 12: at each, the same cells updated
    over the same pending times as the oracle's trigger decides from the
    GPU's own last sub-steps, the others bitwise untouched."""
    d = synth.column_1x32()
    o = oracle_mod.Oracle(d)
    M = 12
    dtg = d.t_span / M
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(4000)
    y = g.state(d.rho0)
    dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    pend = np.zeros(d.n_cells)
    S = d.rho0.sum(1)
    n_skipped = 0
    for _ in range(M):
        y0, dt_prev = y.cpu().numpy(), dt.cpu().numpy()
        st = g.subcycle(y, dtg, dt)
        assert st["status"] == 0 and st["n_failed"] == 0
        exp = o.subcycle(y0, pend, dt_prev, dtg, log_cap=4000)
        due = exp["spans"] > 0
        pend = g.pending().cpu().numpy()
        assert np.array_equal(pend, exp["pending"])
        out = y.cpu().numpy()
        n, logs = rec["n"].cpu().numpy(), rec["dt"].cpu().numpy()
        assert np.array_equal(n > 0, due) and st["accepted"] == n.sum()
        assert np.array_equal(out[~due], y0[~due])
        assert np.array_equal(dt.cpu().numpy()[~due], dt_prev[~due])
        assert np.allclose(log_sums(logs, n)[due], exp["spans"][due], rtol=1e-12)
        if precision == "fp64":
            assert np.array_equal(n, exp["n_log"])
            for c in np.flatnonzero(due):
                assert np.allclose(logs[c, :n[c]], exp["log"][c, :n[c]], rtol=1e-9, atol=0)
            check_fp64(out, exp["rho"], S)
        else:
            want = o.replay(y0, logs, n)
            check_mixed(out[due], want[due], S[due])
        n_skipped += int((~due).sum())
    assert n_skipped > 0                          # the trigger held some cells back


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subcycle_with_nothing_due(coag_mod, precision):
    """A global step far below every cell's last sub-step updates no cell:
    the integration runs over an empty work list and only the pending times
    grow; resetting clears them."""
    d = synth.make_disc(1, 37, 17, 1e-5, 0.1, 10.0, 10.0, 50.0, seed=9)
    g = coag_mod.Coag(d, precision)
    y = g.state(d.rho0)
    dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    g.subcycle(y, d.t_span, dt)                   # every cell: no sub-step yet
    assert np.all(g.pending().cpu().numpy() == 0.0)
    y1, dt1 = y.clone(), dt.clone()
    tiny = 1e-6 * float(dt.min())
    st = g.subcycle(y, tiny, dt)
    assert st["status"] == 0 and st["accepted"] == 0 and st["rejected"] == 0
    assert torch.equal(y, y1) and torch.equal(dt, dt1)
    assert np.all(g.pending(reset=True).cpu().numpy() == tiny)
    assert np.all(g.pending().cpu().numpy() == 0.0)
