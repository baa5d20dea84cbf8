"""Pins of the oracle's vertically integrated kernel (Sec. 5.1).

For the comparison with a surface-density code the paper divides the
collision kernel by sqrt(2 pi (h_i^2 + h_j^2)), the grains forming Gaussian
layers of scale heights h, and sets their vertical relative velocity from
the terminal settling velocities at Z = h.  The pins:
- the scale heights' limits (well mixed for St << alpha, settled as
  H sqrt(alpha / St) for St >> alpha);
- for kernels that do not depend on height, the vertically integrated
  right-hand side equals the height integral of the volume right-hand side
  over the Gaussian layers (the defining property of the factor);
- the settling velocities equal those of the volume form at Z = h;
- a full integration conserves mass and grows grains.
"""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

from test_oracle_rhs import gross_flux


def ring(**kw):
    d = synth.ring_20au()
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_scale_heights_limits(oracle_mod):
    d = ring()
    H = d.extra["H"][0]
    al = d.alpha[0]
    cp = oracle_mod.Oracle(d).cell_physics(0)
    St, h = cp["St"], cp["h"]
    assert np.all(np.diff(h) < 0) and np.all(h <= H)
    # well mixed below alpha, settled above it, each to first order in the
    # small ratio
    small = St < 1e-2 * al
    big = St > 1e2 * al
    assert small.sum() > 10 and big.sum() > 10
    assert np.all(np.abs(h[small] / H - 1) <= 0.5 * St[small] / al)
    assert np.all(np.abs(h[big] / (H * np.sqrt(al / St[big])) - 1) <= 0.5 * al / St[big])
    # the volume form has no layers
    assert np.all(oracle_mod.Oracle(ring(vertical=0)).cell_physics(0)["h"] == 0.0)


@pytest.mark.parametrize("kmode,const", [(synth.KERNEL_CONSTANT, 1e-6), (synth.KERNEL_ADDITIVE, 1e-2)])
@pytest.mark.parametrize("fmode", [synth.FRAG_NONE, synth.FRAG_ALL])
def test_rhs_is_height_integral_of_volume_rhs(oracle_mod, kmode, const, fmode):
    """sum_ij C n_i n_j K / sqrt(2 pi (h_i^2 + h_j^2)) with n = Sigma / m is
    the z-integral of the same bilinear form over n_i(z) = Sigma_i / (m_i
    sqrt(2 pi) h_i) exp(-z^2 / 2 h_i^2), for any height-independent K."""
    N = 24
    d = synth.make_ring_disc(1, N, 1e-5, 1.0, 20.0, 20.0, 1.0, alpha=1e-3, v_frag=100.0)
    d.kernel_mode, d.kernel_const, d.frag_mode = kmode, const / (1.0 if kmode == 1 else d.m[0]), fmode
    rng = np.random.default_rng(5)
    sig = d.rho0.copy()
    sig[0] = rng.uniform(0.1, 1.0, N) * 1e-3
    ov = oracle_mod.Oracle(d)
    h = ov.cell_physics(0)["h"]
    want = ov.rhs(sig)[0]
    # volume form at heights z_q, trapezoid rule (spectrally accurate for
    # these Gaussians) over +-14 of the largest scale height
    L = 14.0 * h.max()
    z = np.linspace(-L, L, 4001)
    dz = z[1] - z[0]
    vol = d.subset(np.zeros(z.size, dtype=int))
    vol.vertical = 0
    vol.Z = np.zeros(z.size)
    rho = sig[0][None, :] / (np.sqrt(2 * np.pi) * h[None, :]) * np.exp(-0.5 * (z[:, None] / h[None, :]) ** 2)
    got = oracle_mod.Oracle(vol).rhs(rho).sum(0) * dz
    # rounding of the literal mass bookkeeping scales with the gross flux
    # (sweep-up pairs of the additive kernel cancel to ~1e-16 of it)
    G = gross_flux(ov, d, sig)[0]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-13 * G)


def test_settling_at_own_scale_height(oracle_mod):
    """Each grain settles as it would at Z = h in the volume form, up to the
    O((h/R)^2) difference between the mid-plane and the spherical Omega."""
    d = ring()
    cp = oracle_mod.Oracle(d).cell_physics(0)
    h, vz = cp["h"], cp["vZ"]
    N = d.n_bins
    vol = d.subset(np.zeros(N, dtype=int))
    vol.vertical = 0
    vol.Z = h.copy()
    ov = oracle_mod.Oracle(vol)
    ref = np.array([ov.cell_physics(k)["vZ"][k] for k in range(N)])
    assert np.all(vz < 0)
    hR = (h / d.R[0]) ** 2
    assert np.all(np.abs(vz / ref - 1) <= 2.0 * hR + 1e-14)


def test_vertical_step_conserves_mass_and_grows(oracle_mod):
    d = ring()
    res = oracle_mod.Oracle(d).step(d.rho0, d.t_span)
    assert np.all(res["status"] == 0)
    S = d.rho0.sum(1)
    assert np.allclose(res["rho"].sum(1), S, rtol=1e-11)
    a = d.extra["a"]
    assert res["rho"][0, a > 1.2e-4].sum() > 0.5 * S[0]      # MRN starts below 1 um


def vi_adj_disc(vdust=False):
    # three rings over 0.1-10 um with strong fragmentation (v_frag 1 cm/s),
    # so that the turbulence, settling and layer-thickness derivatives all
    # carry weight; a spread initial state
    d = synth.make_ring_disc(3, 14, 1e-5, 1e-3, 10.0, 30.0, 300.0, alpha=2e-3, v_frag=1.0, seed=7)
    x = synth.random_state(d, seed=8, spread=2) / (0.01 * d.rho_gas[:, None])   # rows sum to 1
    d.rho0 = np.ascontiguousarray(x * d.rho0.sum(1, keepdims=True))
    if vdust:
        rng = np.random.default_rng(4)
        d.v_dust = rng.standard_normal((3, d.n_cells, d.n_bins)) * 30.0
    return d


@pytest.mark.parametrize("vdust", [False, True])
def test_vertical_adjoint_matches_finite_differences(oracle_mod, vdust):
    """Gradients of L = sum w Sigma(T) after the oracle's own step sequence
    with respect to alpha (which now also moves the scale heights, the
    settling velocities and the layer factor), v_frag and the initial
    surface densities, against central differences of the replay."""
    d = vi_adj_disc(vdust)
    o = oracle_mod.Oracle(d)
    ref = o.step(d.rho0, d.t_span, log_cap=4000)
    hs, n_h = ref["log"], ref["n_log"]
    w = np.random.default_rng(2).standard_normal((d.n_cells, d.n_bins)) / d.rho0.sum(1, keepdims=True)
    g_rho0, g_alpha, g_vf = o.vjp(d.rho0, hs, n_h, w)

    def L_of(mod):
        dd = vi_adj_disc(vdust)
        mod(dd)
        return float((w * oracle_mod.Oracle(dd).replay(dd.rho0, hs, n_h)).sum())

    for c in range(d.n_cells):
        e = 1e-5 * d.alpha[c]
        fd = (L_of(lambda dd: dd.alpha.__setitem__(c, dd.alpha[c] + e))
              - L_of(lambda dd: dd.alpha.__setitem__(c, dd.alpha[c] - e))) / (2 * e)
        assert g_alpha[c] == pytest.approx(fd, rel=1e-5, abs=1e-6 * abs(g_alpha).max())
    e = 1e-5 * d.v_frag
    fd = (L_of(lambda dd: setattr(dd, "v_frag", dd.v_frag + e))
          - L_of(lambda dd: setattr(dd, "v_frag", dd.v_frag - e))) / (2 * e)
    assert g_vf == pytest.approx(fd, rel=1e-6)
    for c, k in ((0, 0), (1, 5), (2, 13)):
        e = 1e-5 * max(d.rho0[c, k], 1e-3 * d.rho0[c].sum())
        rp, rm = d.rho0.copy(), d.rho0.copy()
        rp[c, k] += e
        rm[c, k] -= e
        fd = (float((w * o.replay(rp, hs, n_h)).sum()) - float((w * o.replay(rm, hs, n_h)).sum())) / (2 * e)
        assert g_rho0[c, k] == pytest.approx(fd, rel=2e-6, abs=1e-6 * abs(g_rho0).max())
    # the layer terms matter: dropping them would change the alpha gradient
    assert np.abs(g_alpha).max() > 0
