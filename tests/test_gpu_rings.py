"""Shared-memory ring depths of the mixed kernel (mixed_tile_stages,
mixed_k_stages): the depth of the mapping-tile and K-table rings changes how
far the copies run ahead of the tensor cores, not the arithmetic, so every
depth that fits must give the automatic choice's results bitwise, with the
per-slot state in shared memory or in the device workspace; a request that
fits no cluster size is refused at init."""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "column_1x32_N50": lambda: synth.column_1x32(),
    "N40_4736_cells": lambda: synth.make_disc(74, 64, 40, 1e-5, 1.0, 5.0, 100.0, 50.0, seed=5),
    "N100_1024_cells": lambda: synth.make_disc(16, 64, 100, 1e-5, 10.0, 5.0, 100.0, 100.0, seed=5, rho_pert=0.1),
}


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def make(coag_mod, d, P, sb, ks):
    try:
        return coag_mod.Coag(d, "mixed", mixed_cluster=P, mixed_tile_stages=sb, mixed_k_stages=ks)
    except coag_mod.CoagError as e:
        assert e.status == coag_mod.EINVAL
        return None


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("P", [1, 2, 4])
def test_ring_depths_do_not_change_results(coag_mod, case, P):
    d = CASES[case]()
    ref = coag_mod.Coag(d, "mixed", mixed_cluster=P)
    if ref.mixed_cluster()[0] != P:
        pytest.skip("this size does not fit P CTAs per group")
    yr = ref.state(d.rho0)
    sr = ref.step(yr, d.t_span)
    assert sr["status"] == 0
    rho = synth.random_state(d, seed=21)
    fr = ref.rhs(ref.state(rho)).cpu().numpy()
    tried = 0
    placements = set()
    for sb, ks in [(2, 1), (2, 4), (3, 1), (1, 2), (4, 2)]:
        g = make(coag_mod, d, P, sb, ks)
        if g is None:
            continue
        if g.mixed_cluster()[0] != P:
            g.close()
            continue
        got_sb, got_ks, smem = g.mixed_rings()
        assert (got_sb, got_ks) == (sb, ks)
        placements.add(smem)
        y = g.state(d.rho0)
        st = g.step(y, d.t_span)
        assert st["status"] == 0 and st["accepted"] == sr["accepted"] and st["rejected"] == sr["rejected"]
        assert torch.equal(y, yr)
        assert np.array_equal(g.rhs(g.state(rho)).cpu().numpy(), fr)
        tried += 1
        g.close()
    assert tried >= 1
    ref.close()


def test_state_moves_to_the_workspace_when_the_rings_take_its_room(coag_mod):
    """100 bins, clusters of 4: automatically two tile and two K stages with
    the state in shared memory; four K stages leave no room for it."""
    d = CASES["N100_1024_cells"]()
    a = coag_mod.Coag(d, "mixed", mixed_cluster=4)
    assert a.mixed_cluster()[0] == 4
    assert a.mixed_rings() == (2, 2, 1)
    b = coag_mod.Coag(d, "mixed", mixed_cluster=4, mixed_tile_stages=2, mixed_k_stages=4)
    assert b.mixed_rings() == (2, 4, 0)
    ya, yb = a.state(d.rho0), b.state(d.rho0)
    assert a.step(ya, d.t_span)["status"] == 0 and b.step(yb, d.t_span)["status"] == 0
    assert torch.equal(ya, yb)
    a.close()
    b.close()


def test_rings_that_fit_no_cluster_size_are_refused(coag_mod):
    d = CASES["N100_1024_cells"]()
    with pytest.raises(coag_mod.CoagError) as e:
        coag_mod.Coag(d, "mixed", mixed_tile_stages=4, mixed_k_stages=4)
    assert e.value.status == coag_mod.EINVAL
    assert b"do not fit" in coag_mod.lib().cudisc_coag_last_error(None)
