"""GPU parity of the vertically integrated kernel mode (Sec. 5.1) against the
FP64 CPU oracle, through the C ABI.

Kernel tables and right-hand sides carry the volume form's tolerances: 1e-12
(FP64) and 2e-6 / 3e-5 (FP32 K / K p_frag); right-hand sides 1e-10 (FP64)
and 3e-6 of the gross flux (mixed).  Integrations over 1e4 yr reach the
coagulation-fragmentation balance, where the explicit integrator amplifies
rounding-level differences (see long_run_bound below).
"""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

from long_run import long_run_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def packed(full):
    N = full.shape[1]
    ii, jj = np.tril_indices(N)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    return full[:, ii[order], jj[order]]


def gross(o, d, rho):
    K, _, _ = o.kernel()
    n = rho / d.m
    return (d.m * n * np.einsum("cik,ci->ck", K, n)).sum(1)


CASES = {
    "ring_20au_N150": lambda: synth.ring_20au(),
    "rings_37_N60": lambda: synth.make_ring_disc(37, 60, 1e-5, 1.0, 5.0, 100.0, 1e4, seed=3),
    "rings_9_N17_vdust": None,
}


def make(case):
    if case == "rings_9_N17_vdust":
        d = synth.make_ring_disc(9, 17, 1e-5, 0.1, 10.0, 50.0, 1e3, seed=4)
        rng = np.random.default_rng(6)
        d.v_dust = rng.standard_normal((3, d.n_cells, d.n_bins)) * 10.0
        return d
    return CASES[case]()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vertical_kernel_matches_oracle(coag_mod, oracle_mod, case, precision):
    d = make(case)
    K, pf, _ = oracle_mod.Oracle(d).kernel()
    g = coag_mod.Coag(d, precision)
    Kg, KFg = (x.cpu().numpy() for x in g.get_kernel())
    Ko, KFo = packed(K), packed(K * pf)
    if precision == "fp64":
        assert np.allclose(Kg, Ko, rtol=1e-12, atol=0)
        assert np.allclose(KFg, KFo, rtol=1e-9, atol=1e-14 * Ko.max())
    else:
        assert np.allclose(Kg, Ko, rtol=2e-6, atol=0)
        assert np.all(np.abs(KFg - KFo) <= 3e-5 * np.abs(KFo) + 2e-6 * Ko)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vertical_rhs_matches_oracle(coag_mod, oracle_mod, case, precision):
    d = make(case)
    sig = synth.random_state(d, seed=31)
    o = oracle_mod.Oracle(d)
    ref = o.rhs(sig)
    G = gross(o, d, sig)
    g = coag_mod.Coag(d, precision)
    out = g.rhs(g.state(sig)).cpu().numpy()
    tol = 1e-10 if precision == "fp64" else 3e-6
    err = np.abs(out - ref) / G[:, None]
    assert err.max() < tol, err.max()


def test_vertical_step_fp64_short_span(coag_mod, oracle_mod):
    """100 yr (before the fragmentation balance): the oracle's own step
    sequence and states to 1e-10."""
    d = synth.make_ring_disc(37, 60, 1e-5, 1.0, 5.0, 100.0, 100.0, seed=3)
    ref = oracle_mod.Oracle(d).step(d.rho0, d.t_span, log_cap=4000)
    g = coag_mod.Coag(d, "fp64")
    rec = g.set_records(4000)
    y = g.state(d.rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0 and st["n_failed"] == 0
    assert np.array_equal(rec["n"].cpu().numpy(), ref["n_log"])
    S = d.rho0.sum(1)
    r = np.abs(y.cpu().numpy() - ref["rho"]) / (1e-10 * np.abs(ref["rho"]) + 1e-20 * S[:, None])
    assert r.max() <= 1.0, r.max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["ring_20au_N150", "rings_37_N60", "rings_4096_N100"])
def test_vertical_long_run_replayed_by_oracle(coag_mod, oracle_mod, precision, case):
    """1e4 yr: the oracle replays the GPU's accepted steps on sampled cells;
    every bin within long_run_bound, and the mixed path's bins within the
    strict 1e-5 bound but for a few percent."""
    d = synth.rings_4096() if case == "rings_4096_N100" else make(case)
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(4000)
    y = g.state(d.rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0 and st["n_failed"] == 0
    assert st["mass_err_max"] < (1e-12 if precision == "fp64" else 1e-9)
    n = rec["n"].cpu().numpy()
    assert st["accepted"] == n.sum() and n.min() >= 1
    cells = np.unique(np.linspace(0, d.n_cells - 1, min(12, d.n_cells)).astype(int))
    ds = d.subset(cells)
    y0, strict, bound = long_run_bound(oracle_mod, ds, d.rho0[cells], rec["dt"].cpu().numpy()[cells],
                                       n[cells], precision)
    dev = np.abs(y.cpu().numpy()[cells] - y0)
    assert np.all(dev <= bound), (dev / bound).max()
    assert np.mean(dev <= strict) >= 0.95
    assert np.allclose(rec["dt"].cpu().numpy().sum(1), d.t_span, rtol=1e-12)
