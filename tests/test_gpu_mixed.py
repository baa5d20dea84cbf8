"""GPU parity of the mixed-precision (tcgen05 TF32 split) path against the
FP64 CPU oracle, through the C ABI.

Tolerances, derived from the arithmetic: each contraction term carries the
FP32 rounding of x_i x_j K and K itself (~1e-7) and the TF32 hi/lo split
(2^-21 of the generated operand, 2^-22 of the mapping coefficients), and the
tensor core accumulates in FP32, so a right-hand side
agrees with the oracle to a few 1e-7 of the cell's gross collision flux
(checked at 3e-6).  Integrated states: |d rho_k| <= 1e-5 |rho_k| + 1e-10 S,
i.e. 1e-5 relative with the paper's absolute tolerance (1e-10 of the cell's
dust mass S) as the floor.  Growth-front and trace bins below ~1e-6 S are fed
by net fluxes 1e4-1e5 times smaller than their gross fluxes, so a right-hand
side error of a few 1e-7 of the gross flux shows up there as an absolute
error of a few 1e-11 S.  Total mass is conserved to 1e-9.
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


def check_state(out, ref, S, rel=1e-5, atol_rel=1e-10):
    """|d rho_k| <= 1e-5 |rho_k| + 1e-10 S per bin: the stated relative
    tolerance with the paper's absolute tolerance (1e-10 sum_k rho_k) as the
    floor, the same atol + rtol |y| form as the integrator's error scale."""
    r = np.abs(out - ref) / (rel * np.abs(ref) + atol_rel * S[:, None])
    assert r.max() <= 1.0, f"error {r.max():.3f} x (1e-5 |rho| + 1e-10 S)"
    return r.max()


CASES = {
    # slot counts per CTA of 16, 32, 64, 128 and the refill path
    "N2_one_cell": lambda: synth.make_disc(1, 1, 2, 1e-5, 1e-3, 10.0, 10.0, 50.0),
    "N17_37_cells": lambda: synth.make_disc(1, 37, 17, 1e-5, 0.1, 10.0, 10.0, 50.0, seed=9),
    "column_1x32_N50": lambda: synth.column_1x32(),
    "N40_4736_cells": lambda: synth.make_disc(74, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5),
    "N24_9000_cells": lambda: synth.make_disc(100, 90, 24, 1e-5, 0.1, 5.0, 100.0, 20.0, seed=6),
    "N20_20000_cells_refill": lambda: synth.make_disc(200, 100, 20, 1e-5, 0.1, 5.0, 100.0, 20.0, seed=7),
    "N128_5_cells": lambda: synth.make_disc(1, 5, 128, 1e-5, 10.0, 10.0, 10.0, 20.0),
    # bins past 128: MMA N of 144 and 160 (0.1 um - 1 m for 150 bins)
    "N129_3_cells": lambda: synth.make_disc(1, 3, 129, 1e-5, 10.0, 10.0, 10.0, 20.0, seed=13),
    "N150_9_cells": lambda: synth.make_disc(3, 3, 150, 1e-5, 100.0, 5.0, 100.0, 20.0, alpha=1e-4,
                                            v_frag=1000.0, seed=14),
    # the largest bin count the library takes (MMA N of 160 per tile)
    "N160_4_cells": lambda: synth.make_disc(2, 2, 160, 1e-5, 300.0, 5.0, 100.0, 20.0, alpha=1e-4,
                                            v_frag=1000.0, seed=15),
}
SMALL = ["N2_one_cell", "N17_37_cells", "column_1x32_N50", "N128_5_cells", "N129_3_cells",
         "N150_9_cells", "N160_4_cells"]


def sample_of(d, k=24):
    return np.unique(np.linspace(0, d.n_cells - 1, min(k, d.n_cells)).astype(int))


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_mixed_matches_oracle(coag_mod, oracle_mod, case):
    d = CASES[case]()
    rho = synth.random_state(d, seed=21)
    g = coag_mod.Coag(d, "mixed")
    out = g.rhs(g.state(rho)).cpu().numpy()
    cells = sample_of(d)
    ds = d.subset(cells)
    o = oracle_mod.Oracle(ds)
    ref = o.rhs(rho[cells])
    G = gross(o, ds, rho[cells])
    err = np.abs(out[cells] - ref) / G[:, None]
    assert err.max() < 3e-6, err.max()
    # the FP64 mass budget makes every right-hand side conserve mass
    assert np.all(np.abs(out.sum(1)) <= 1e-13 * np.abs(out).sum(1) + 1e-300)


@pytest.mark.parametrize("case", SMALL)
def test_kernel_build_fp32_matches_oracle(coag_mod, oracle_mod, case):
    d = CASES[case]()
    o = oracle_mod.Oracle(d)
    K, pf, _ = o.kernel()
    g = coag_mod.Coag(d, "mixed")
    Kg, KFg = (x.cpu().numpy() for x in g.get_kernel())
    Ko, KFo = packed(K), packed(K * pf)
    assert np.allclose(Kg, Ko, rtol=2e-6, atol=0)
    # p_frag = (1 + x) exp(-x) turns a relative error e of dv into ~2 x^2 e / (1 + x)
    assert np.all(np.abs(KFg - KFo) <= 3e-5 * np.abs(KFo) + 2e-6 * Ko)


@pytest.mark.parametrize("case", ["N17_37_cells", "column_1x32_N50", "N128_5_cells", "N150_9_cells"])
def test_replay_mixed_matches_oracle(coag_mod, oracle_mod, case):
    """The oracle's own accepted step sequence replayed by both sides."""
    d = CASES[case]()
    o = oracle_mod.Oracle(d)
    ref = o.step(d.rho0, d.t_span, log_cap=4000)
    want = o.replay(d.rho0, ref["log"], ref["n_log"])
    g = coag_mod.Coag(d, "mixed")
    y = g.state(d.rho0)
    g.replay(y, torch.as_tensor(ref["log"], device="cuda"), torch.as_tensor(ref["n_log"], device="cuda"))
    S = d.rho0.sum(1)
    check_state(y.cpu().numpy(), want, S)
    assert np.abs(y.cpu().numpy().sum(1) / S - 1).max() < 1e-9


@pytest.mark.parametrize("case", ["column_1x32_N50", "N40_4736_cells", "N20_20000_cells_refill"])
def test_free_running_mixed_step(coag_mod, oracle_mod, case):
    """Free-running adaptive step: the oracle replays the GPU's own accepted
    step sequence (decisions near E = 1 may differ between precisions)."""
    d = CASES[case]()
    g = coag_mod.Coag(d, "mixed")
    rec = g.set_records(3000)
    y = g.state(d.rho0)
    dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    st = g.step(y, d.t_span, dt)
    assert st["status"] == 0 and st["n_failed"] == 0
    assert st["mass_err_max"] < 1e-9
    n = rec["n"].cpu().numpy()
    assert n.max() <= 3000 and n.min() >= 1
    assert st["accepted"] == n.sum()
    cells = sample_of(d, 16)
    ds = d.subset(cells)
    want = oracle_mod.Oracle(ds).replay(d.rho0[cells], rec["dt"].cpu().numpy()[cells], n[cells])
    S = d.rho0[cells].sum(1)
    check_state(y.cpu().numpy()[cells], want, S)
    # every cell ran to t_span: its accepted steps add up to it
    assert np.allclose(rec["dt"].cpu().numpy().sum(1), d.t_span, rtol=1e-12)


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_cluster_sizes_match_oracle(coag_mod, oracle_mod, cluster):
    """Every split of a slot group's pass over a cluster of CTAs (the partial
    sums and stage inputs they exchange): right-hand sides, and a
    free-running step with slot refills (4736 cells, more than the slots of
    clusters of 4 or 8) replayed by the oracle on sampled cells."""
    d = CASES["N40_4736_cells"]()
    g = coag_mod.Coag(d, "mixed", mixed_cluster=cluster)
    P, groups = g.mixed_cluster()
    assert P == cluster and groups >= 1
    rho = synth.random_state(d, seed=23)
    out = g.rhs(g.state(rho)).cpu().numpy()
    cells = sample_of(d, 12)
    ds = d.subset(cells)
    o = oracle_mod.Oracle(ds)
    err = np.abs(out[cells] - o.rhs(rho[cells])) / gross(o, ds, rho[cells])[:, None]
    assert err.max() < 3e-6, err.max()
    rec = g.set_records(3000)
    y = g.state(d.rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0 and st["n_failed"] == 0
    assert st["mass_err_max"] < 1e-9
    n = rec["n"].cpu().numpy()
    assert st["accepted"] == n.sum()
    want = o.replay(d.rho0[cells], rec["dt"].cpu().numpy()[cells], n[cells])
    check_state(y.cpu().numpy()[cells], want, d.rho0[cells].sum(1))
    assert np.allclose(rec["dt"].cpu().numpy().sum(1), d.t_span, rtol=1e-12)


def test_automatic_cluster_choice(coag_mod):
    """Few cells per slot: the pass is split over more CTAs; many cells: one
    CTA per group (its exchanges cost more than the split saves)."""
    few = coag_mod.Coag(CASES["N17_37_cells"](), "mixed")
    many = coag_mod.Coag(CASES["N20_20000_cells_refill"](), "mixed")
    assert few.mixed_cluster()[0] >= 2
    assert many.mixed_cluster()[0] <= 2
    assert coag_mod.Coag(CASES["N17_37_cells"](), "fp64").mixed_cluster() == (0, 0)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_empty_cell_passes_through(coag_mod, oracle_mod, precision):
    """A cell without dust (atol = 0, zero right-hand side) takes one step of
    t_span, stays empty and leaves the other cells as the oracle has them."""
    d = CASES["N17_37_cells"]()
    rho0 = d.rho0.copy()
    rho0[[0, 5, 36]] = 0.0
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(3000)
    y = g.state(rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0 and st["n_failed"] == 0
    out = y.cpu().numpy()
    n = rec["n"].cpu().numpy()
    assert np.all(out[[0, 5, 36]] == 0.0) and np.all(n[[0, 5, 36]] == 1)
    cells = [1, 2, 20, 35]
    want = oracle_mod.Oracle(d.subset(cells)).replay(rho0[cells], rec["dt"].cpu().numpy()[cells], n[cells])
    check_state(out[cells], want, rho0[cells].sum(1))


def test_mixed_maxsteps_status(coag_mod):
    d = CASES["N17_37_cells"]()
    d.max_substeps = 4
    g = coag_mod.Coag(d, "mixed")
    st = g.step(g.state(d.rho0), d.t_span, check=False)
    assert st["status"] == coag_mod.EMAXSTEPS and st["n_failed"] == d.n_cells


def test_full_size_grid_mixed_rhs_sampled(coag_mod, oracle_mod):
    """128 x 64 cells x 100 bins in the launch configuration the benchmark
    uses; sampled cells against the oracle."""
    d = synth.grid_128x64()
    rho = synth.random_state(d, seed=5)
    g = coag_mod.Coag(d, "mixed")
    out = g.rhs(g.state(rho)).cpu().numpy()
    cells = np.arange(0, d.n_cells, 331)
    ds = d.subset(cells)
    o = oracle_mod.Oracle(ds)
    ref = o.rhs(rho[cells])
    err = np.abs(out[cells] - ref) / gross(o, ds, rho[cells])[:, None]
    assert err.max() < 3e-6, err.max()


def test_full_size_large_grid_mixed_rhs_sampled(coag_mod, oracle_mod):
    """512 x 256 cells x 150 bins (0.1 um - 1 m): kernel build and the mixed
    right-hand side of all 131072 cells; sampled cells against the oracle."""
    d = synth.grid_512x256()
    rho = synth.random_state(d, seed=17)
    g = coag_mod.Coag(d, "mixed")
    out = g.rhs(g.state(rho)).cpu().numpy()
    g.close()
    cells = np.arange(0, d.n_cells, 8191)
    ds = d.subset(cells)
    o = oracle_mod.Oracle(ds)
    ref = o.rhs(rho[cells])
    err = np.abs(out[cells] - ref) / gross(o, ds, rho[cells])[:, None]
    assert err.max() < 3e-6, err.max()
    assert np.isfinite(out).all()


def test_full_size_fp64_step_conserves_mass(coag_mod):
    """With the double-double mapping coefficients the FP64 path conserves
    total mass to ~1e-13 over 1e4 yr of the 128 x 64 x 100 workload."""
    d = synth.grid_128x64()
    g = coag_mod.Coag(d, "fp64")
    y = g.state(d.rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0
    assert st["mass_err_max"] < 1e-12, st["mass_err_max"]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_size_long_run_sampled_cells(coag_mod, oracle_mod, precision):
    """The benchmark's step at full size and in its launch configuration:
    all 8192 cells over 1e4 yr; on 12 sampled cells the oracle replays the
    GPU's accepted steps.  Every bin within the long-run bound (see
    long_run.py), at least 97 % within 1e-5 |rho| + 1e-10 S, mass to 1e-9."""
    d = synth.grid_128x64()
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(2000)
    y = g.state(d.rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0 and st["n_failed"] == 0
    assert st["mass_err_max"] < (1e-12 if precision == "fp64" else 1e-9)
    n = rec["n"].cpu().numpy()
    assert n.max() <= 2000 and st["accepted"] == n.sum()
    cells = np.arange(0, d.n_cells, 683)[:12]
    y0, strict, bound = long_run_bound(oracle_mod, d.subset(cells), d.rho0[cells],
                                       rec["dt"].cpu().numpy()[cells], n[cells], precision)
    dev = np.abs(y.cpu().numpy()[cells] - y0)
    assert np.all(dev <= bound), (dev / bound).max()
    assert np.mean(dev <= strict) >= 0.97


def test_full_size_large_grid_short_integration_replayed(coag_mod, oracle_mod):
    """512 x 256 cells x 150 bins in the large-grid launch configuration (one
    CTA per group, two tile stages, one K stage, the K tables prefetched into
    L2 since they exceed it): all 131072 cells over 30 yr, short of the
    coagulation-fragmentation balance; on sampled cells the oracle replays the
    GPU's accepted steps and every bin agrees to 1e-5 |rho| + 1e-10 S."""
    d = synth.grid_512x256()
    d.t_span = 30.0 * synth.CONST["yr"]
    g = coag_mod.Coag(d, "mixed")
    assert g.mixed_cluster()[0] == 1 and g.mixed_rings()[:2] == (2, 1)
    rec = g.set_records(1000)
    y = g.state(d.rho0)
    st = g.step(y, d.t_span)
    assert st["status"] == 0 and st["n_failed"] == 0 and st["mass_err_max"] < 1e-9
    n = rec["n"].cpu().numpy()
    assert n.max() <= 1000 and st["accepted"] == n.sum()
    cells = np.arange(0, d.n_cells, 16381)
    o = oracle_mod.Oracle(d.subset(cells))
    dts = rec["dt"][torch.as_tensor(cells, device=rec["dt"].device)].cpu().numpy()
    want = o.replay(d.rho0[cells], dts, n[cells])
    S = d.rho0[cells].sum(1)
    got = y.cpu().numpy()[cells]
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-10 * S[:, None])
    g.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_non_finite_cell_fails_alone(coag_mod, precision):
    """A NaN in one cell's state: that cell ends with ENONFINITE, every other
    cell succeeds and equals a clean integration bitwise (a slot's generated
    operand rows reach only that slot's outputs)."""
    d = synth.make_disc(4, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5)
    bad = 77
    rho = d.rho0.copy()
    rho[bad, 3] = np.nan
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(4000)
    y = g.state(rho)
    st = g.step(y, d.t_span, check=False)
    assert st["status"] == coag_mod.ENONFINITE and st["n_failed"] == 1
    status = rec["status"].cpu().numpy()
    ok = np.arange(d.n_cells) != bad
    assert status[bad] == coag_mod.ENONFINITE and np.all(status[ok] == 0)
    g.set_records(0)
    y2 = g.state(d.rho0)
    assert g.step(y2, d.t_span)["status"] == 0
    assert np.array_equal(y.cpu().numpy()[ok], y2.cpu().numpy()[ok])
    g.close()
