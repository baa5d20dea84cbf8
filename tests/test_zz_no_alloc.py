"""The allocation-free step entry point, through the C ABI.

cudisc_coag_step_static_scratch serves callers that cannot allocate device
memory where they integrate (for example a code whose device memory belongs
to its own pool allocator): its integrator scratch is a fixed device array
inside the library.  Its results must match cudisc_coag_step within the
mixed-path tolerance, call after call, although every call reuses the same
array.  This file is collected last on purpose.
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


def within(out, ref, S):
    """|d rho| <= 1e-5 |rho| + 1e-10 S, the tolerance of the mixed-path tests."""
    return (np.abs(out - ref) <= 1e-5 * np.abs(ref) + 1e-10 * S[:, None]).all()


def _column():
    return synth.column_1x32(), {}, False


def _small_disc():
    return synth.make_disc(1, 37, 17, 1e-5, 0.1, 10.0, 10.0, 50.0, seed=9), {}, False


def _global_state_disc():
    # 100 bins with one CTA per slot group: the per-slot state (64 slots x 5
    # x 100 x 4 B per group) does not fit beside the rings in shared memory,
    # so it lives in the scratch array; 1024 cells make 128 groups, 16.4 MB
    d = synth.make_disc(16, 64, 100, 1e-5, 10.0, 5.0, 100.0, 300.0, seed=5, rho_pert=0.1)
    return d, {"mixed_cluster": 1}, True


@pytest.mark.parametrize("make", [_column, _small_disc, _global_state_disc])
def test_static_scratch_step_matches_step_twice(coag_mod, make):
    d, over, in_array = make()
    g = coag_mod.Coag(d, "mixed", **over)
    scratch = coag_mod.cudisc_coag_scratch_bytes(g.ctx)
    if in_array:
        # the per-slot state is in global scratch: these calls read and write the array
        assert 0 < scratch <= 16 << 20, scratch
    else:
        assert scratch == 0      # shared memory holds it; the array is not touched
    S = d.rho0.sum(1)
    ref = g.state(d.rho0)
    dt_ref = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    st = g.step(ref, d.t_span, dt_ref)
    assert st["status"] == 0
    ref = ref.cpu().numpy()
    for _ in range(2):
        y = g.state(d.rho0)
        dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
        st2, s = coag_mod.cudisc_coag_step_static_scratch(g.ctx, y.data_ptr(), d.t_span, dt.data_ptr())
        assert st2 == 0
        assert s.accepted == st["accepted"] and s.mass_err_max < 1e-9
        assert s.elapsed_ms > 0.0
        assert within(y.cpu().numpy(), ref, S)
        assert np.allclose(dt.cpu().numpy(), dt_ref.cpu().numpy(), rtol=1e-12)
    g.close()


def test_static_scratch_rejects_oversized_and_wrong_precision(coag_mod):
    # one CTA per group: 148 groups x 64 slots x 5 x 100 bins x 4 B > 16 MiB
    big = synth.grid_128x64()
    g = coag_mod.Coag(big, "mixed", mixed_cluster=1)
    assert g.mixed_cluster() == (1, 148)
    assert coag_mod.cudisc_coag_scratch_bytes(g.ctx) == 148 * 64 * 5 * 100 * 4
    y = g.state(big.rho0)
    st, _ = coag_mod.cudisc_coag_step_static_scratch(g.ctx, y.data_ptr(), big.t_span, None, check=False)
    assert st == coag_mod.ENOTSUP
    assert b"static" in coag_mod.lib().cudisc_coag_last_error(g.ctx)
    g.close()
    small = synth.column_1x32()
    g64 = coag_mod.Coag(small, "fp64")
    y = g64.state(small.rho0)
    st, _ = coag_mod.cudisc_coag_step_static_scratch(g64.ctx, y.data_ptr(), small.t_span, None, check=False)
    assert st == coag_mod.EINVAL
