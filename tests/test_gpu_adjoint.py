"""GPU adjoint (cudisc_coag_vjp) against the FP64 oracle's discrete adjoint,
through the C ABI, on the same frozen step sequences.

Tolerances.  FP64 contexts differentiate the same map as the oracle in the
same precision.  The two differ in how the mapping coefficients are rounded:
double-double on the GPU side, and the literal FP64 expressions in the
oracle.  In the oracle, a pair (i, j) with m_j << m_i forms m_i + m_j and
then subtracts m_i again, so each transposed pair term carries a relative
error up to eps m_i / m_j.
  - Grids spanning m_max / m_min <= 1e6 keep that floor below 1e-10, and the
    gradients agree to 1e-9 of the cell's largest component.
  - Full-range grids (0.1 um - 1 cm, m_max / m_min ~ 1e15) put the oracle's
    floor near 1e-4 of the largest component (measured: 2e-4 on the
    50-bin column).  There the GPU's FP64 adjoint is pinned instead by
    central differences of the GPU's own FP64 forward and by the dot-product
    identity; the oracle comparison uses 1e-3.
Mixed contexts run the same FP64 adjoint on their own map, whose kernel
tables come from the FP32 builder: K within 2e-6 and K p_frag within 3e-5 of
the FP64 tables.  Propagated through the integration, those perturbations
move the gradients by ~1e-5 of the cell's largest component.  The check is
1e-4, against either the oracle (narrow grids) or the FP64 context's adjoint
(any grid).  The scalar gradients (alpha, v_frag) get 5e-4.  They are signed
sums over every pair of every transposed evaluation, and in a fragmentation
equilibrium those sums cancel to ~1e-1 of their gross, which scales up the
same table perturbations.
"""
import numpy as np
import pytest

from paper_2402_18471_b300 import synth

from test_oracle_vertical import vi_adj_disc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def adj_disc():
    # 0.1 - 10 um, strong fragmentation; the oracle's own finite-difference pin disc
    d = synth.make_disc(1, 4, 14, 1e-5, 1e-3, 10.0, 10.0, 3000.0, alpha=2e-3, v_frag=1.0, seed=3)
    d.rho0 = synth.random_state(d, seed=8, spread=2)
    return d


def column8():
    d = synth.column_1x32().subset(list(range(0, 32, 4)))
    d.t_span = 300.0 * synth.CONST["yr"]
    return d


def wide_alpha():
    # 24 cells, 40 bins over 0.1 um - 1 mm, alpha spread 0.3 dex, fragmentation at 1 m/s
    return synth.make_disc(4, 6, 40, 1e-5, 0.1, 5.0, 50.0, 500.0, alpha=1e-3, alpha_dex=0.3,
                           v_frag=100.0, seed=11)


def narrow_alpha():
    # 24 cells, 40 bins over 0.1 - 10 um, alpha spread 0.3 dex, v_frag 3 cm/s
    d = synth.make_disc(4, 6, 40, 1e-5, 1e-3, 5.0, 50.0, 1000.0, alpha=1e-3, alpha_dex=0.3,
                        v_frag=3.0, seed=12)
    d.rho0 = synth.random_state(d, seed=13, spread=3)
    return d


NARROW = {"adj_disc_N14": adj_disc, "narrow_alpha_N40": narrow_alpha,
          # vertically integrated kernel (Sec. 5.1): alpha also moves the
          # scale heights, the settling and the layer factor
          "vertical_rings3_N14": lambda: vi_adj_disc(False),
          "vertical_rings3_N14_vdust": lambda: vi_adj_disc(True)}
WIDE = {"column8_N50": column8, "wide_alpha_N40": wide_alpha}
CASES = {**NARROW, **WIDE}


def oracle_log(oracle_mod, d):
    o = oracle_mod.Oracle(d)
    r = o.step(d.rho0, d.t_span, log_cap=4000)
    assert (r["status"] == 0).all()
    return o, r["log"], r["n_log"]


def weights(d, seed=3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((d.n_cells, d.n_bins)) / d.rho0.sum(1, keepdims=True)


def gpu_vjp(coag_mod, d, precision, w, hs, n_h):
    g = coag_mod.Coag(d, precision)
    g0, ga, gv = g.vjp(g.state(d.rho0), torch.as_tensor(w, device="cuda"),
                       torch.as_tensor(hs, device="cuda"), torch.as_tensor(n_h, device="cuda"))
    out = g0.cpu().numpy(), ga.cpu().numpy(), float(gv.cpu()[0])
    g.close()
    return out


def check(got, want, rel, what, rel_scalar=None):
    g0, ga, gv = got
    w0, wa, wv = want
    rs = 2 * rel if rel_scalar is None else rel_scalar
    scale = np.abs(w0).max(1, keepdims=True)
    e0 = (np.abs(g0 - w0) / scale).max()
    ea = np.abs(ga - wa).max() / np.abs(wa).max()
    ev = abs(gv - wv) / abs(wv)
    assert e0 <= rel, f"{what}: grad_rho0 error {e0:.3e} of the cell's largest component"
    assert ea <= rs, f"{what}: grad_alpha error {ea:.3e}"
    assert ev <= rs, f"{what}: grad_vfrag error {ev:.3e}"
    return e0, ea, ev


# (precision, grad_rho0 tolerance, scalar-gradient tolerance)
PRECISIONS = [("fp64", 1e-9, 2e-9), ("mixed", 1e-4, 5e-4)]


@pytest.mark.parametrize("case", list(NARROW))
@pytest.mark.parametrize("precision,rel,rel_s", PRECISIONS)
def test_vjp_matches_oracle(coag_mod, oracle_mod, case, precision, rel, rel_s):
    d = NARROW[case]()
    o, hs, n_h = oracle_log(oracle_mod, d)
    w = weights(d)
    want = o.vjp(d.rho0, hs, n_h, w)
    got = gpu_vjp(coag_mod, d, precision, w, hs, n_h)
    check(got, want, rel, f"{case}/{precision}", rel_s)


@pytest.mark.parametrize("case", list(WIDE))
def test_vjp_full_range_grids(coag_mod, oracle_mod, case):
    """0.1 um - 1 cm grids: FP64 GPU adjoint against the oracle within the
    oracle's rounding floor, FP32 adjoint against the FP64 GPU adjoint."""
    d = WIDE[case]()
    o, hs, n_h = oracle_log(oracle_mod, d)
    w = weights(d)
    want = o.vjp(d.rho0, hs, n_h, w)
    g64 = gpu_vjp(coag_mod, d, "fp64", w, hs, n_h)
    g32 = gpu_vjp(coag_mod, d, "mixed", w, hs, n_h)
    check(g64, want, 1e-3, f"{case}/fp64 vs oracle")
    check(g32, g64, 1e-4, f"{case}/mixed vs fp64", 5e-4)


@pytest.mark.parametrize("precision,rel,rel_s", PRECISIONS)
def test_vjp_checkpoint_segment_edges(coag_mod, oracle_mod, precision, rel, rel_s):
    """Step counts on and around the 16-substep checkpoint boundaries, and
    zero steps (the identity), in one launch."""
    d = synth.make_disc(1, 7, 20, 1e-5, 1e-3, 10.0, 10.0, 3e4, v_frag=3.0, seed=4)
    d.rho0 = synth.random_state(d, seed=5, spread=3)
    o, hs, n_h = oracle_log(oracle_mod, d)
    counts = np.array([0, 1, 15, 16, 17, 32, 33])
    assert (n_h >= counts).all()
    w = weights(d, seed=9)
    want = o.vjp(d.rho0, hs, counts, w)
    got = gpu_vjp(coag_mod, d, precision, w, hs, counts)
    assert np.array_equal(got[0][0], w[0]) and got[1][0] == 0.0
    keep = np.arange(1, d.n_cells)
    check((got[0][keep], got[1][keep], got[2]), (want[0][keep], want[1][keep], want[2]), rel,
          f"segments/{precision}", rel_s)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vjp_internal_forward_equals_recorded(coag_mod, precision):
    """hs = NULL integrates rho0 adaptively inside the call; that is the same
    step sequence a cudisc_coag_step call records, so the gradients match
    bit for bit."""
    d = CASES["column8_N50"]()
    g = coag_mod.Coag(d, precision)
    rec = g.set_records(4000)
    y = g.state(d.rho0)
    g.step(y, d.t_span)
    g.set_records(0)
    w = torch.as_tensor(weights(d), device="cuda")
    a = g.vjp(g.state(d.rho0), w, rec["dt"], rec["n"])
    b = g.vjp(g.state(d.rho0), w, t_span=d.t_span)
    for x, z in zip(a, b):
        assert torch.equal(x, z)
    assert g.timings()["vjp_ms"] > 0


@pytest.mark.parametrize("case", ["adj_disc_N14", "column8_N50"])
def test_vjp_fp64_matches_gpu_finite_differences(coag_mod, case):
    """Central differences of the GPU's own FP64 replay (relative step 1e-5)
    in alpha, v_frag and the initial densities of the largest and smallest
    bins, against the GPU adjoint; and the dot-product identity
    <J u, w> = <u, J^T w> along a random direction u."""
    d = CASES[case]()
    g = coag_mod.Coag(d, "fp64")
    rec = g.set_records(4000)
    g.step(g.state(d.rho0), d.t_span)
    g.set_records(0)
    hs, n_h = rec["dt"].clone(), rec["n"].clone()
    w = torch.as_tensor(weights(d), device="cuda")
    g0, ga, gv = g.vjp(g.state(d.rho0), w, hs, n_h)

    def L(alpha=None, vf=None):
        if alpha is not None:
            g.set_alpha(alpha)
        if vf is not None:
            g.set_v_frag(vf)
        g.build_kernel()
        y = g.state(d.rho0)
        g.replay(y, hs, n_h)
        return float((w * y).sum())

    ga = ga.cpu().numpy()
    for c in range(min(d.n_cells, 4)):
        e = 1e-5 * d.alpha[c]
        ap, am = d.alpha.copy(), d.alpha.copy()
        ap[c] += e
        am[c] -= e
        fd = (L(alpha=ap) - L(alpha=am)) / (2 * e)
        assert ga[c] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(ga).max())
    L(alpha=d.alpha)
    e = 1e-5 * d.v_frag
    fd = (L(vf=d.v_frag + e) - L(vf=d.v_frag - e)) / (2 * e)
    assert float(gv.cpu()[0]) == pytest.approx(fd, rel=1e-5)
    L(vf=d.v_frag)

    def Lr(r0):
        y = g.state(r0)
        g.replay(y, hs, n_h)
        return float((w * y).sum())

    g0 = g0.cpu().numpy()
    for k in (0, d.n_bins - 1, d.n_bins // 2):
        e = 1e-5 * max(d.rho0[0, k], 1e-3 * d.rho0[0].sum())
        rp, rm = d.rho0.copy(), d.rho0.copy()
        rp[0, k] += e
        rm[0, k] -= e
        fd = (Lr(rp) - Lr(rm)) / (2 * e)
        assert g0[0, k] == pytest.approx(fd, rel=2e-6, abs=1e-6 * np.abs(g0[0]).max())
    u = np.random.default_rng(5).standard_normal(d.rho0.shape) * d.rho0
    eps = 1e-5
    lhs = (Lr(d.rho0 + eps * u) - Lr(d.rho0 - eps * u)) / (2 * eps)
    assert lhs == pytest.approx(float((u * g0).sum()), rel=1e-7)


def test_autograd_function(coag_mod):
    """coag_step as a torch.autograd.Function: backward gives the adjoint of
    the recorded step sequence for rho0, alpha and v_frag."""
    d = CASES["wide_alpha_N40"]()
    g = coag_mod.Coag(d, "mixed")
    rho0 = torch.as_tensor(d.rho0, device="cuda").requires_grad_(True)
    alpha = torch.as_tensor(d.alpha, device="cuda").requires_grad_(True)
    vf = torch.tensor(d.v_frag, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.as_tensor(weights(d), device="cuda")
    y = coag_mod.coag_step(rho0, alpha, vf, g, d.t_span)
    (w * y).sum().backward()
    rec = g.set_records(4000)
    g.step(g.state(d.rho0), d.t_span)
    g.set_records(0)
    g0, ga, gv = g.vjp(g.state(d.rho0), w, rec["dt"], rec["n"])
    assert torch.equal(rho0.grad, g0)
    assert torch.equal(alpha.grad, ga)
    assert vf.grad.shape == vf.shape and float(vf.grad) == float(gv[0])


def test_adjoint_workload_sampled(coag_mod, oracle_mod):
    """64 R x 32 Z x 80 bins over 2000 yr, alpha lognormal 0.3 dex, the loss
    being the mass of grains below 10 um above Z = H: the mixed (FP32)
    adjoint on every cell, sampled cells against the oracle's adjoint of the
    GPU's own step sequence."""
    d = synth.adjoint_64x32()
    w = synth.adjoint_loss_weights(d)
    g = coag_mod.Coag(d, "mixed")
    rec = g.set_records(4000)
    st = g.step(g.state(d.rho0), d.t_span)
    assert st["status"] == 0
    g.set_records(0)
    n = rec["n"].cpu().numpy()
    assert n.max() <= 4000
    g0, ga, gv = g.vjp(g.state(d.rho0), torch.as_tensor(w, device="cuda"), rec["dt"], rec["n"])
    g0, ga = g0.cpu().numpy(), ga.cpu().numpy()
    assert np.isfinite(g0).all() and np.isfinite(ga).all() and np.isfinite(float(gv.cpu()[0]))
    # FP32 adjoint against the FP64 GPU adjoint of the same map, every cell
    g64 = coag_mod.Coag(d, "fp64")
    h0, ha, hv = g64.vjp(g64.state(d.rho0), torch.as_tensor(w, device="cuda"), rec["dt"], rec["n"])
    h0, ha = h0.cpu().numpy(), ha.cpu().numpy()
    hot = np.flatnonzero(w.sum(1) > 0)
    scale = np.abs(h0[hot]).max(1, keepdims=True)
    assert (np.abs(g0[hot] - h0[hot]) / scale).max() <= 1e-4
    assert np.abs(ga - ha).max() <= 5e-4 * np.abs(ha).max()
    assert abs(float(gv.cpu()[0]) - float(hv.cpu()[0])) <= 5e-4 * abs(float(hv.cpu()[0]))
    # and the FP64 adjoint against the oracle on sampled cells (full-range floor)
    cells = hot[np.linspace(0, len(hot) - 1, 8).astype(int)]
    ds = d.subset(cells)
    want = oracle_mod.Oracle(ds).vjp(ds.rho0, rec["dt"].cpu().numpy()[cells], n[cells], w[cells])
    e0 = (np.abs(h0[cells] - want[0]) / np.abs(want[0]).max(1, keepdims=True)).max()
    ea = (np.abs(ha[cells] - want[1]) / np.abs(want[1]).max()).max()
    assert e0 <= 1e-3, e0
    assert ea <= 2e-3, ea


def df_vs_fp64(coag_mod, d, precision, w, hs, n_h):
    """The same context's adjoint in FP64 and then in double-float."""
    g = coag_mod.Coag(d, precision)
    args = (g.state(d.rho0), torch.as_tensor(w, device="cuda"), torch.as_tensor(hs, device="cuda"),
            torch.as_tensor(n_h, device="cuda"))
    out = []
    for p in ("fp64", "double_float", "fp64"):
        g.set_adjoint_precision(p)
        g0, ga, gv = g.vjp(*args)
        out.append((g0.cpu().numpy(), ga.cpu().numpy(), float(gv.cpu()[0])))
    g.close()
    return out


# Double-float adjoint (cudisc_coag_set_adjoint_precision): each per-pair
# term carries ~2^-46 of its size instead of FP64's 2^-53, i.e. ~2e2 times the
# FP64 adjoint's rounding; the sums whose cancellation the tolerances above
# allow for scale it the same way.  Against the FP64 GPU adjoint of the same
# map: 1e-7 of the cell's largest component, 1e-6 for the scalar gradients.
@pytest.mark.parametrize("case", list(CASES))
def test_double_float_adjoint_matches_fp64(coag_mod, oracle_mod, case):
    d = CASES[case]()
    _, hs, n_h = oracle_log(oracle_mod, d)
    w = weights(d)
    first, df, again = df_vs_fp64(coag_mod, d, "fp64", w, hs, n_h)
    # switching back rebuilds the FP64 tables: bitwise the first result
    assert all(np.array_equal(a, b) for a, b in zip(first[:2], again[:2])) and first[2] == again[2]
    check(df, first, 1e-7, f"{case}/double_float", 1e-6)


def test_double_float_adjoint_on_the_adjoint_workload(coag_mod):
    """64 R x 32 Z x 80 bins over 2000 yr with the mixed forward's records:
    the double-float adjoint of the mixed context against its FP64 adjoint
    on every cell."""
    d = synth.adjoint_64x32()
    w = synth.adjoint_loss_weights(d)
    g = coag_mod.Coag(d, "mixed")
    rec = g.set_records(4000)
    assert g.step(g.state(d.rho0), d.t_span)["status"] == 0
    g.set_records(0)
    res = []
    for p in ("fp64", "double_float"):
        g.set_adjoint_precision(p)
        g0, ga, gv = g.vjp(g.state(d.rho0), torch.as_tensor(w, device="cuda"), rec["dt"], rec["n"])
        res.append((g0.cpu().numpy(), ga.cpu().numpy(), float(gv.cpu()[0])))
    (h0, ha, hv), (g0, ga, gv) = res
    assert np.isfinite(g0).all() and np.isfinite(ga).all() and np.isfinite(gv)
    hot = np.flatnonzero(w.sum(1) > 0)
    scale = np.abs(h0[hot]).max(1, keepdims=True)
    assert (np.abs(g0[hot] - h0[hot]) / scale).max() <= 1e-7
    assert np.abs(ga - ha).max() <= 1e-6 * np.abs(ha).max()
    assert abs(gv - hv) <= 1e-6 * abs(hv)
