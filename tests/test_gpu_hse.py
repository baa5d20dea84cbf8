"""GPU parity of the hydrostatic-equilibrium gas density (Sec. 3.5) against
the FP64 CPU oracle, through the C ABI.

Tolerance 1e-12 relative per cell: both sides evaluate the same FP64
formulas; the GPU multiplies the ratios in a different order (a warp scan
in passes of 32 cells) and sums omega V in a different order, each a few
ulp per cell.
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


def gpu_hse(coag_mod, inp):
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    out = coag_mod.hse_rho_gas(dev(inp["R"]), dev(inp["Z"]), dev(inp["T"]), dev(inp["V"]),
                               dev(inp["R_edges"]), dev(inp["Sigma_g"]), inp["mu"], inp["m_H"],
                               inp["k_B"], inp["GM"])
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_cols(hse_mod, inp, cols):
    rows = []
    for i in cols:
        sub = {k: inp[k] for k in ("mu", "m_H", "k_B", "GM")}
        for k in ("R", "Z", "T", "V"):
            sub[k] = inp[k][i:i + 1]
        sub["R_edges"] = inp["R_edges"][i:i + 2]
        sub["Sigma_g"] = inp["Sigma_g"][i:i + 1]
        rows.append(hse_mod.hse_rho_gas(**sub)[0])
    return np.array(rows)


@pytest.mark.parametrize("n_R,n_Z", [(1, 1), (1, 17), (5, 32), (33, 100), (3, 300)])
@pytest.mark.parametrize("t_rise", [0.0, 3.0])
def test_hse_matches_oracle(coag_mod, n_R, n_Z, t_rise):
    from oracle import hse
    d = synth.make_disc(n_R, n_Z, 4, 1e-5, 1e-4, 5.0, 100.0, 1.0, seed=2)
    inp = synth.hse_inputs(d, t_rise=t_rise)
    got = gpu_hse(coag_mod, inp)
    want = hse.hse_rho_gas(**inp)
    assert np.all(got > 0)
    assert np.allclose(got, want, rtol=1e-12, atol=0)


def test_hse_full_size_large_grid_sampled(coag_mod):
    """512 x 256 cells: every column on the GPU, sampled columns against the
    oracle, the normalisation of every column."""
    from oracle import hse
    d = synth.grid_512x256()
    inp = synth.hse_inputs(d, t_rise=2.0)
    got = gpu_hse(coag_mod, inp)
    cols = np.arange(0, d.n_R, 37)
    assert np.allclose(got[cols], oracle_cols(hse, inp, cols), rtol=1e-12, atol=0)
    RdR = 0.5 * (inp["R_edges"][1:] ** 2 - inp["R_edges"][:-1] ** 2)
    assert np.allclose((got * inp["V"]).sum(1), inp["Sigma_g"] * RdR, rtol=1e-12)


def test_hse_density_feeds_the_kernel_build(coag_mod, oracle_mod):
    """The gas density computed on the GPU, written into the array a context
    reads, then the kernel rebuilt: K as the oracle has it for that gas."""
    d = synth.make_disc(4, 16, 30, 1e-5, 1.0, 5.0, 100.0, 100.0, seed=3)
    inp = synth.hse_inputs(d, t_rise=1.0)
    g = coag_mod.Coag(d, "fp64")
    rho_g = gpu_hse(coag_mod, inp).reshape(-1)
    g._keep["rho_gas"].copy_(torch.as_tensor(rho_g, device="cuda"))
    g.build_kernel()
    K, _ = g.get_kernel()
    d2 = d.subset(np.arange(d.n_cells))
    d2.rho_gas = rho_g.copy()
    Ko, _, _ = oracle_mod.Oracle(d2).kernel()
    ii, jj = np.tril_indices(d.n_bins)
    order = np.argsort(ii * (ii + 1) // 2 + jj)
    assert np.allclose(K.cpu().numpy(), Ko[:, ii[order], jj[order]], rtol=1e-12)
