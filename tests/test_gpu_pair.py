"""The mixed kernel in CTA pairs (mixed_pair = 2): two CTAs share each M = 256
tensor-core MMA (tcgen05 cta_group::2), each keeping half of every mapping
tile.  With P pairs per cluster each slot group's blocks are split between P
CTAs exactly as with P single CTAs per group, and every row of an MMA is
the same dot product whatever M, so pair mode must reproduce single mode
bitwise; against the oracle it is held to the mixed path's tolerances."""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "N2_one_cell": lambda: synth.make_disc(1, 1, 2, 1e-5, 1e-3, 10.0, 10.0, 50.0),
    "N17_37_cells": lambda: synth.make_disc(1, 37, 17, 1e-5, 0.1, 10.0, 10.0, 50.0, seed=9),
    "column_1x32_N50": lambda: synth.column_1x32(),
    "N40_4736_cells": lambda: synth.make_disc(74, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5),
    "N128_5_cells": lambda: synth.make_disc(1, 5, 128, 1e-5, 10.0, 10.0, 10.0, 20.0),
    "N100_1024_cells": lambda: synth.make_disc(16, 64, 100, 1e-5, 10.0, 5.0, 100.0, 100.0, seed=5, rho_pert=0.1),
}


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def pair_and_single(coag_mod, d, P):
    gp = coag_mod.Coag(d, "mixed", mixed_cluster=P, mixed_pair=2)
    gs = coag_mod.Coag(d, "mixed", mixed_cluster=P, mixed_pair=1)
    return gp, gs


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("P", [1, 2, 4])
def test_pair_rhs_equals_single_bitwise(coag_mod, oracle_mod, case, P):
    d = CASES[case]()
    gp, gs = pair_and_single(coag_mod, d, P)
    if gp.mixed_pair() == 0 or gp.mixed_cluster()[0] != P or gs.mixed_cluster()[0] != P:
        pytest.skip("this size does not fit P pairs")
    rho = synth.random_state(d, seed=21)
    fp = gp.rhs(gp.state(rho)).cpu().numpy()
    fs = gs.rhs(gs.state(rho)).cpu().numpy()
    assert np.array_equal(fp, fs)
    gp.close()
    gs.close()


@pytest.mark.parametrize("case", ["column_1x32_N50", "N40_4736_cells", "N100_1024_cells"])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_pair_step_equals_single_bitwise(coag_mod, case, P):
    """Free-running adaptive integrations: the same accepted steps and end
    states (cells take slots in a different order, but a cell's arithmetic
    does not depend on its slot)."""
    d = CASES[case]()
    gp, gs = pair_and_single(coag_mod, d, P)
    if gp.mixed_pair() == 0 or gp.mixed_cluster()[0] != P:
        pytest.skip("this size does not fit P pairs")
    yp, ys = gp.state(d.rho0), gs.state(d.rho0)
    dp = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    ds = torch.zeros_like(dp)
    sp = gp.step(yp, d.t_span, dp)
    ss = gs.step(ys, d.t_span, ds)
    assert sp["status"] == 0 and ss["status"] == 0
    assert sp["accepted"] == ss["accepted"] and sp["rejected"] == ss["rejected"]
    assert torch.equal(yp, ys) and torch.equal(dp, ds)
    gp.close()
    gs.close()


def test_pair_replay_matches_oracle(coag_mod, oracle_mod):
    d = CASES["column_1x32_N50"]()
    o = oracle_mod.Oracle(d)
    ref = o.step(d.rho0, d.t_span, log_cap=4000)
    want = o.replay(d.rho0, ref["log"], ref["n_log"])
    g = coag_mod.Coag(d, "mixed", mixed_pair=2)
    assert g.mixed_pair() == 1
    y = g.state(d.rho0)
    g.replay(y, torch.as_tensor(ref["log"], device="cuda"), torch.as_tensor(ref["n_log"], device="cuda"))
    S = d.rho0.sum(1)
    got = y.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-10 * S[:, None])
    assert np.abs(got.sum(1) / S - 1).max() < 1e-9


def test_full_size_bench_grid_in_pairs(coag_mod):
    """The 128 x 64 x 100 bench grid over 1e4 yr in pair mode: every cell
    succeeds, mass holds, and the result equals single mode with the same
    number of CTAs per group bitwise."""
    d = synth.grid_128x64()
    gp, gs = pair_and_single(coag_mod, d, 2)
    assert gp.mixed_pair() == 1 and gp.mixed_cluster()[0] == 2 and gs.mixed_cluster()[0] == 2
    yp, ys = gp.state(d.rho0), gs.state(d.rho0)
    sp = gp.step(yp, d.t_span)
    ss = gs.step(ys, d.t_span)
    assert sp["status"] == 0 and sp["n_failed"] == 0 and sp["mass_err_max"] < 1e-9
    assert sp["accepted"] == ss["accepted"]
    assert torch.equal(yp, ys)


def test_pair_request_falls_back_above_128_bins(coag_mod):
    d = synth.make_disc(1, 3, 129, 1e-5, 10.0, 10.0, 10.0, 20.0, seed=13)
    g = coag_mod.Coag(d, "mixed", mixed_pair=2)
    assert g.mixed_pair() == 0
    y = g.state(d.rho0)
    assert g.step(y, d.t_span)["status"] == 0


@pytest.mark.parametrize("P", [1, 2])
def test_pair_wait_runs_out_then_recovers(coag_mod, P):
    d = synth.make_disc(4, 64, 50, 1e-5, 1.0, 5.0, 40.0, 20.0, seed=31)
    g = coag_mod.Coag(d, "mixed", mixed_cluster=P, mixed_pair=2)
    assert g.mixed_pair() == 1
    ref = g.state(d.rho0)
    assert g.step(ref, d.t_span)["status"] == 0
    coag_mod.cudisc_coag_set_fault_injection(g.ctx, 2_000_000, 1)
    y = g.state(d.rho0)
    status, _ = coag_mod.cudisc_coag_step(g.ctx, y.data_ptr(), d.t_span, None, check=False)
    assert status == coag_mod.ECUDA
    coag_mod.cudisc_coag_set_fault_injection(g.ctx, 0, 0)
    y = g.state(d.rho0)
    assert g.step(y, d.t_span)["status"] == 0
    assert torch.equal(y, ref)
    g.close()


@pytest.mark.parametrize("P,pair", [(4, 1), (8, 1), (4, 2)])
def test_refilled_cells_reproducible(coag_mod, P, pair):
    """Cells that take a slot freed during the launch land in a slot that
    depends on timing; their results must not (each slot's partial rows are
    added in member order)."""
    d = CASES["N40_4736_cells"]()
    g = coag_mod.Coag(d, "mixed", mixed_cluster=P, mixed_pair=pair)
    groups = g.mixed_cluster()[1]
    assert groups * 64 < d.n_cells                # some cells are refills
    rho = synth.random_state(d, seed=21)
    outs = [g.rhs(g.state(rho)).cpu().numpy() for _ in range(3)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    g.close()
