"""GPU parity of the dust source update and CFL step (Sec. 3.1) with the FP64
oracle, through the C ABI.  Both sides evaluate the same FP64 formulas; the
GPU forms the per-cell factors once and multiplies by reciprocals, a few ulp
per element: 1e-12 of each field's scale."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G_M = 6.674e-8 * 1.989e33
AU = 1.496e13


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def inputs(n_s, n_c, seed):
    rng = np.random.default_rng(seed)
    R = AU * rng.uniform(5, 100, n_c)
    Z = R * rng.uniform(0.0, 0.2, n_c)
    rho_g = 10.0 ** rng.uniform(-16, -10, n_c)
    c_s = rng.uniform(1e4, 1e5, n_c)
    v_g = np.stack([rng.normal(0, 1e3, n_c), np.sqrt(G_M / R) * (1 - 1e-3), rng.normal(0, 10, n_c)])
    a = 10.0 ** np.linspace(-5, 1, n_s)
    P = np.empty((4, n_s, n_c))
    P[0] = 10.0 ** rng.uniform(-20, -12, (n_s, n_c))
    P[1] = rng.normal(0, 1e3, (n_s, n_c))
    P[2] = np.sqrt(G_M / R)[None, :] * (1 + rng.normal(0, 1e-3, (n_s, n_c)))
    P[3] = rng.normal(0, 1e2, (n_s, n_c))
    Q = np.stack([P[0], P[0] * P[1], P[0] * P[2] * R[None, :], P[0] * P[3]])
    Q = Q * (1 + rng.normal(0, 1e-3, Q.shape))          # as after a transport half-step
    return Q, P, R, Z, rho_g, c_s, v_g, a


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def close(got, want):
    scale = np.abs(want).max(axis=(1, 2), keepdims=True)
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want) + 1e-14 * scale)


@pytest.mark.parametrize("n_s,n_c", [(1, 1), (7, 33), (40, 1000), (3, 257)])
@pytest.mark.parametrize("h", [3e7, 3e9])
def test_source_update_matches_oracle(coag_mod, n_s, n_c, h):
    from oracle import dust
    Q, P, R, Z, rho_g, c_s, v_g, a = inputs(n_s, n_c, seed=n_s * 1000 + n_c)
    want = dust.source_update(Q, P, h, R, Z, rho_g, c_s, v_g, a, 1.6, G_M)
    q = dev(Q)
    coag_mod.dust_source_update(q, dev(P), h, dev(R), dev(Z), dev(rho_g), dev(c_s), dev(v_g), dev(a), 1.6, G_M)
    torch.cuda.synchronize()
    close(q.cpu().numpy(), want)


def test_source_update_bench_grid_sampled(coag_mod):
    """8192 cells x 100 species; the oracle on sampled cells (cells are
    independent)."""
    from oracle import dust
    n_s, n_c = 100, 8192
    Q, P, R, Z, rho_g, c_s, v_g, a = inputs(n_s, n_c, seed=7)
    q = dev(Q)
    coag_mod.dust_source_update(q, dev(P), 1e9, dev(R), dev(Z), dev(rho_g), dev(c_s), dev(v_g), dev(a), 1.6, G_M)
    got = q.cpu().numpy()
    cells = np.arange(0, n_c, 409)
    want = dust.source_update(Q[:, :, cells], P[:, :, cells], 1e9, R[cells], Z[cells], rho_g[cells],
                              c_s[cells], v_g[:, cells], a, 1.6, G_M)
    close(got[:, :, cells], want)


@pytest.mark.parametrize("n_s,n_c", [(1, 1), (5, 300), (100, 8192)])
def test_cfl_matches_oracle(coag_mod, n_s, n_c):
    from oracle import dust
    _, P, R, _, _, c_s, _, _ = inputs(n_s, n_c, seed=11)
    rng = np.random.default_rng(12)
    P[1, rng.random((n_s, n_c)) < 0.1] = 0.0        # zero velocities impose no limit
    dR = R * 0.02
    dZ = R * 0.003
    nu = 1e-3 * c_s * c_s / np.sqrt(G_M / R ** 3)
    Sc = rng.uniform(0.5, 2.0, n_s)
    want = dust.cfl_dt(P[1], P[3], dR, dZ, nu, Sc)
    got = float(coag_mod.dust_cfl_dt(dev(P), dev(dR), dev(dZ), dev(nu), dev(Sc)).cpu()[0])
    assert got == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("where", ["v_R", "v_Z", "Sc", "dR", "nu"])
def test_cfl_flags_inputs_outside_its_domain(coag_mod, where):
    """One non-finite velocity, or a non-positive Sc or dR, or a negative nu,
    gives NaN rather than a finite step from the remaining elements."""
    _, P, R, _, _, c_s, _, _ = inputs(6, 700, seed=21)
    dR = R * 0.02
    dZ = R * 0.003
    nu = 1e-3 * c_s * c_s / np.sqrt(G_M / R ** 3)
    Sc = np.ones(6)
    ok = float(coag_mod.dust_cfl_dt(dev(P), dev(dR), dev(dZ), dev(nu), dev(Sc)).cpu()[0])
    assert np.isfinite(ok) and ok > 0
    if where == "v_R":
        P[1, 3, 411] = np.nan
    elif where == "v_Z":
        P[3, 0, 699] = np.inf
    elif where == "Sc":
        Sc[2] = -1.0
    elif where == "dR":
        dR[5] = 0.0
    else:
        nu[300] = -nu[300]
    out = coag_mod.dust_cfl_dt(dev(P), dev(dR), dev(dZ), dev(nu), dev(Sc)).cpu().numpy()
    assert np.isnan(out[0]) and np.isnan(out[1])
