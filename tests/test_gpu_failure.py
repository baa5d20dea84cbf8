"""The mixed kernel's failure path, made to happen without faulting the GPU.

Every wait of the mixed integration kernel on another role's progress is
bounded.  Through the test hook cudisc_coag_set_fault_injection the limit is
shortened to ~1 ms and the bulk-copy producer issues nothing, so that every
consumer's wait runs out: the call must return CUDISC_ECUDA with the
"bounded device wait ran out" message, and the same context must then
integrate normally, bitwise equal to a run that never failed."""
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


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_wait_runs_out_then_the_context_recovers(coag_mod, cluster):
    d = synth.make_disc(4, 64, 50, 1e-5, 1.0, 5.0, 40.0, 20.0, seed=31)   # 256 cells, 50 bins
    g = coag_mod.Coag(d, "mixed", mixed_cluster=cluster)
    assert g.mixed_cluster()[0] == cluster
    ref = g.state(d.rho0)
    st = g.step(ref, d.t_span)
    assert st["status"] == 0
    ref = ref.cpu().numpy()

    coag_mod.cudisc_coag_set_fault_injection(g.ctx, 2_000_000, 1)
    y = g.state(d.rho0)
    status, _ = coag_mod.cudisc_coag_step(g.ctx, y.data_ptr(), d.t_span, None, check=False)
    assert status == coag_mod.ECUDA
    assert b"bounded device wait ran out" in coag_mod.lib().cudisc_coag_last_error(g.ctx)

    coag_mod.cudisc_coag_set_fault_injection(g.ctx, 0, 0)
    y = g.state(d.rho0)
    st2 = g.step(y, d.t_span)
    assert st2["status"] == 0 and st2["accepted"] == st["accepted"]
    assert np.array_equal(y.cpu().numpy(), ref)
    g.close()


def test_fp64_context_ignores_the_hook(coag_mod):
    d = synth.column_1x32()
    g = coag_mod.Coag(d, "fp64")
    coag_mod.cudisc_coag_set_fault_injection(g.ctx, 2_000_000, 1)
    y = g.state(d.rho0)
    assert g.step(y, d.t_span)["status"] == 0
    g.close()
