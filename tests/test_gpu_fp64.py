"""GPU parity of the FP64 path against the FP64 CPU oracle, through the C ABI.

Tolerance (FP64 path): 1e-10 relative per element, with an absolute floor
tied to the cell's gross collision flux (right-hand side) or to the paper's
absolute tolerance 1e-10 sum_k rho_k (states), since single bins can cancel
to zero in exact arithmetic.
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


def packed(full):
    """[c, N, N] -> [c, Np] with p = i (i+1)/2 + j, j <= i."""
    N = full.shape[1]
    ii, jj = np.tril_indices(N)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    return full[:, ii[order], jj[order]]


def gross(o, d, rho):
    K, _, _ = o.kernel()
    n = rho / d.m
    return (d.m * n * np.einsum("cik,ci->ck", K, n)).sum(1)


def small_disc(N=12, cells=5, **kw):
    d = synth.make_disc(1, cells, N, 1e-5, 1.0, 10.0, 10.0, 100.0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


CASES = {
    "column_1x32_N50": lambda: synth.column_1x32(),
    "N2_one_cell": lambda: small_disc(N=2, cells=1),
    "N17_ragged_37_cells": lambda: synth.make_disc(1, 37, 17, 1e-5, 0.1, 10.0, 10.0, 50.0, seed=9),
    "N150_3_cells": lambda: synth.make_disc(1, 3, 150, 1e-5, 100.0, 10.0, 10.0, 100.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_kernel_build_fp64_matches_oracle(coag_mod, oracle_mod, case):
    d = CASES[case]()
    o = oracle_mod.Oracle(d)
    K, pf, _ = o.kernel()
    g = coag_mod.Coag(d, "fp64")
    Kg, KFg = (x.cpu().numpy() for x in g.get_kernel())
    Ko, KFo = packed(K), packed(K * pf)
    assert np.allclose(Kg, Ko, rtol=1e-12, atol=0)
    assert np.allclose(KFg, KFo, rtol=1e-9, atol=1e-14 * Ko.max())


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("fmode,split", [(0, 0), (0, 1), (2, 0), (1, 0)])
def test_rhs_fp64_matches_oracle(coag_mod, oracle_mod, case, fmode, split):
    d = CASES[case]()
    d.frag_mode, d.split_mode = fmode, split
    o = oracle_mod.Oracle(d)
    rho = synth.random_state(d, seed=11)
    ref = o.rhs(rho)
    g = coag_mod.Coag(d, "fp64")
    out = g.rhs(g.state(rho)).cpu().numpy()
    tol = 1e-10 * np.abs(ref) + 1e-13 * gross(o, d, rho)[:, None]
    assert np.all(np.abs(out - ref) <= tol)


def test_rhs_fp64_with_input_dust_velocities(coag_mod, oracle_mod):
    d = synth.column_1x32()
    rng = np.random.default_rng(3)
    d.v_dust = rng.normal(0.0, 30.0, size=(3, d.n_cells, d.n_bins))
    o = oracle_mod.Oracle(d)
    rho = synth.random_state(d, seed=2)
    ref = o.rhs(rho)
    g = coag_mod.Coag(d, "fp64")
    out = g.rhs(g.state(rho)).cpu().numpy()
    assert np.all(np.abs(out - ref) <= 1e-10 * np.abs(ref) + 1e-13 * gross(o, d, rho)[:, None])


def state_close(a, b, S, rel=1e-10):
    return np.abs(a - b) <= rel * np.abs(b) + 1e-10 * rel * S[:, None] * 1e3


def test_step_fp64_free_running_matches_oracle(coag_mod, oracle_mod):
    d = synth.column_1x32()
    o = oracle_mod.Oracle(d)
    ref = o.step(d.rho0, d.t_span, log_cap=4000)
    g = coag_mod.Coag(d, "fp64")
    rec = g.set_records(4000)
    rho = g.state(d.rho0)
    dt = torch.zeros(d.n_cells, dtype=torch.float64, device="cuda")
    st = g.step(rho, d.t_span, dt)
    assert st["status"] == 0 and st["n_failed"] == 0
    assert st["accepted"] == ref["n_acc"].sum() and st["rejected"] == ref["n_rej"].sum()
    assert np.array_equal(rec["n"].cpu().numpy(), ref["n_log"])
    assert np.allclose(rec["dt"].cpu().numpy(), ref["log"], rtol=1e-9, atol=0)
    S = d.rho0.sum(1)
    out = rho.cpu().numpy()
    assert np.all(np.abs(out - ref["rho"]) <= 1e-10 * np.abs(ref["rho"]) + 1e-20 * S[:, None])
    assert st["mass_err_max"] < 1e-13
    assert np.allclose(dt.cpu().numpy(), ref["dt"], rtol=1e-9)


def test_step_fp64_replay_matches_oracle(coag_mod, oracle_mod):
    d = CASES["N17_ragged_37_cells"]()
    o = oracle_mod.Oracle(d)
    ref = o.step(d.rho0, d.t_span, log_cap=3000)
    hs = ref["log"]
    want = o.replay(d.rho0, hs, ref["n_log"])
    g = coag_mod.Coag(d, "fp64")
    rho = g.state(d.rho0)
    g.replay(rho, torch.as_tensor(hs, device="cuda"), torch.as_tensor(ref["n_log"], device="cuda"))
    S = d.rho0.sum(1)
    assert np.all(np.abs(rho.cpu().numpy() - want) <= 1e-10 * np.abs(want) + 1e-20 * S[:, None])


def test_step_fp64_constant_kernel_closed_form(coag_mod):
    """Constant kernel on a linear grid (Sec. 5.1 analytic test) on the GPU."""
    N, m0, N0, K = 64, 2.0 ** -40, 1.0, 1e-6
    d = small_disc(N=N, cells=2)
    d.m, d.me = synth.linear_mass_grid(N, m0)
    d.kernel_mode, d.kernel_const, d.frag_mode = 1, K, 1
    d.rtol, d.atol_rel = 1e-8, 1e-25
    rho0 = np.zeros((2, N)); rho0[:, 0] = N0 * m0
    g = coag_mod.Coag(d, "fp64")
    rho = g.state(rho0)
    st = g.step(rho, 1.0 / (K * N0))
    n = rho.cpu().numpy()[0] / d.m
    k = np.arange(1, N + 1)
    ref = N0 * 0.5 ** (k - 1) / 1.5 ** (k + 1)
    sel = ref > 1e-12
    assert st["status"] == 0
    assert np.allclose(n[sel], ref[sel], rtol=2e-5)


def test_step_fp64_reports_maxsteps(coag_mod):
    d = synth.column_1x32()
    d.max_substeps = 3
    g = coag_mod.Coag(d, "fp64")
    rec = g.set_records(8)
    rho = g.state(d.rho0)
    st = g.step(rho, d.t_span, check=False)
    assert st["status"] == coag_mod.EMAXSTEPS
    assert st["n_failed"] == d.n_cells
    assert np.all(rec["status"].cpu().numpy() == coag_mod.EMAXSTEPS)
    # the context stays usable after a failed call
    d.max_substeps = 10 ** 6
    g2 = coag_mod.Coag(d, "fp64")
    st2 = g2.step(g2.state(d.rho0), 10.0 * synth.CONST["yr"])
    assert st2["status"] == 0


def test_full_size_grid_sampled_cells_fp64(coag_mod, oracle_mod):
    """The 128 x 64 x 100 workload at full size: kernel build and right-hand
    side of every cell on the GPU, checked on a deterministic sample of cells
    against the oracle run on those cells alone (cells are independent)."""
    d = synth.grid_128x64()
    g = coag_mod.Coag(d, "fp64")
    rho = synth.random_state(d, seed=5)
    out = g.rhs(g.state(rho)).cpu().numpy()
    K, KF = g.get_kernel()
    sample = np.arange(0, d.n_cells, 409)
    ds = d.subset(sample)
    o = oracle_mod.Oracle(ds)
    Ko, pfo, _ = o.kernel()
    assert np.allclose(K[sample].cpu().numpy(), packed(Ko), rtol=1e-12)
    ref = o.rhs(rho[sample])
    tol = 1e-10 * np.abs(ref) + 1e-13 * gross(o, ds, rho[sample])[:, None]
    assert np.all(np.abs(out[sample] - ref) <= tol)
