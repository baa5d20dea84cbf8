"""GPU parity of the dust transport step (Sec. 3.1-3.2, Appendix A) with the
FP64 oracle, through the C ABI (cudisc_dust_init / _step).  Both sides are
FP64 and evaluate the same formulas in a different order (the GPU fuses
multiply-adds and builds the stencil coefficients on the device): after a
few steps every field agrees to 1e-11 of that field's largest magnitude."""
import math

import numpy as np
import pytest

from oracle import transport as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AU = 1.495978707e13
G_M = 6.6743e-8 * 1.98847e33


@pytest.fixture(scope="module")
def coag_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18471_b300 import coag
    return coag


def disc_setup(nR, nZ, ns, seed, th1=0.25, R0=5.0, R1=50.0):
    """A thin disc patch: log-spaced radii (au), polar angles 0..th1 above
    the mid-plane, Gaussian gas, near-Keplerian dust with perturbations."""
    rng = np.random.default_rng(seed)
    R_e = AU * np.geomspace(R0, R1, nR + 1)
    th_e = np.linspace(0.0, th1, nZ + 1)
    Rc = 0.5 * (R_e[1:] + R_e[:-1])
    thc = 0.5 * (th_e[1:] + th_e[:-1])
    Z = Rc[:, None] * np.tan(thc)[None, :]
    cs = 1e5 * (Rc / AU / 10.0) ** -0.25
    Om = np.sqrt(G_M / Rc ** 3)
    H = cs / Om
    rho_g = 1e-10 * ((Rc / AU) ** -2.25)[:, None] * np.exp(-0.5 * (Z / H[:, None]) ** 2) * (1 + 0.1 * rng.random((nR, nZ)))
    nu = 1e-3 * (cs * H)[:, None] * np.ones((1, nZ))
    vK = np.sqrt(G_M / Rc)
    P = np.zeros((4, ns, nR, nZ))
    P[0] = 0.01 * rho_g[None] * rng.uniform(0.2, 1.0, (ns, 1, 1)) * (1 + 0.3 * rng.random((ns, nR, nZ)))
    P[1] = -30.0 * rng.random((ns, nR, nZ))
    P[2] = vK[None, :, None] * (1 + 1e-3 * rng.normal(size=(ns, nR, nZ)))
    P[3] = -Z[None] * Om[None, :, None] * 1e-2 * rng.random((ns, nR, nZ))
    Q = np.stack([P[0], P[0] * P[1], P[0] * P[2] * Rc[None, :, None], P[0] * P[3]])
    src = dict(c_s=np.repeat(cs[:, None], nZ, 1), v_g=np.stack([0 * Z, vK[:, None] * np.ones((1, nZ)), 0 * Z]),
               a=np.geomspace(1e-4, 1.0, ns), rho_m=1.6, GM=G_M)
    Sc = rng.uniform(0.7, 1.5, ns)
    return R_e, th_e, Q, rho_g, nu, Sc, src


def compare(got, want, tol=1e-11):
    scale = np.abs(want).max(axis=(2, 3), keepdims=True) + 1e-300
    err = np.abs(got - want) / scale
    assert err.max() <= tol, err.max()
    return err.max()


BCS = {"paper": (T.OUTFLOW, T.OUTFLOW, T.CLOSED, T.OUTFLOW),
       "closed": (T.CLOSED,) * 4,
       "zero": (T.ZERO, T.OUTFLOW, T.CLOSED, T.ZERO)}


@pytest.mark.parametrize("geometry", ["cylindrical", "cartesian"])
@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("diffusion", [True, False])
@pytest.mark.parametrize("sources", [True, False])
def test_steps_match_oracle(coag_mod, geometry, bc, diffusion, sources):
    nR, nZ, ns = 37, 29, 3                       # 1073 cells: several 256-thread blocks and a ragged tail
    R_e, th_e, Q, rho_g, nu, Sc, src = disc_setup(nR, nZ, ns, seed=10 * len(geometry) + list(BCS).index(bc))
    floor = 1e-25
    g = T.Grid(R_e, th_e, geometry=geometry)
    tr = T.Transport(g, rho_g, nu=nu if diffusion else None, Sc=Sc if diffusion else None, bc=BCS[bc],
                     floor=floor, sources=src if sources else None)
    gpu = coag_mod.DustTransport(R_e, th_e, ns, rho_g, nu=nu if diffusion else None, Sc=Sc if diffusion else None,
                                 geometry=geometry, bc=BCS[bc], floor=floor, sources=src if sources else None)
    q = torch.as_tensor(Q, device="cuda").contiguous()
    torch.cuda.synchronize()
    want = Q
    # with sources, also a fraction of the shortest orbital time (gravity
    # changes the velocities within the step; the CFL step of the start state
    # does not see that)
    t_orb = 1.0 / math.sqrt(G_M / R_e[0] ** 3)
    for _ in range(3):
        dt = 0.5 * tr.cfl_dt(want)
        if sources:
            dt = min(dt, 0.02 * t_orb)
        want = tr.step(want, dt)
        gpu.step(q, dt)
    torch.cuda.synchronize()
    compare(q.cpu().numpy(), want)
    gpu.close()


def test_geometry_matches_the_paper_formulas(coag_mod):
    R_e, th_e, Q, rho_g, nu, Sc, src = disc_setup(9, 7, 1, seed=3)
    for geometry in ("cylindrical", "cartesian"):
        g = T.Grid(R_e, th_e, geometry=geometry)
        gpu = coag_mod.DustTransport(R_e, th_e, 1, rho_g, geometry=geometry)
        V, AR, AZ = (x.cpu().numpy() for x in gpu.geometry())
        a = T.NG
        assert np.allclose(V, g.V[a:a + 9, a:a + 7], rtol=1e-14, atol=0)
        assert np.allclose(AR, g.AR[a:a + 10, a:a + 7], rtol=1e-14, atol=0)
        assert np.allclose(AZ, g.AZ[a:a + 9, a:a + 8], rtol=1e-14, atol=0)
        gpu.close()


def test_gaussian_pulse_run_matches_oracle(coag_mod):
    """The paper's advected-diffused pulse (Sec. 3.4) on 48 x 48 cells from
    t = 0.1 to 1 with the oracle's CFL steps: the GPU's end state matches the
    oracle's, so its L2 error against the closed form is the oracle's."""
    N = 48
    R_e = np.geomspace(10.0, 50.0, N + 1)
    th_e = np.linspace(-math.pi / 6, math.pi / 6, N + 1)
    g = T.Grid(R_e, th_e, geometry="cartesian")
    a = T.NG
    x = g.Rc[a:a + N][:, None] * np.ones((1, N))
    y = g.Zc[a:a + N, a:a + N]

    def exact(t):
        return 0.01 + 1.0 / t * np.exp(-((x - 30.0 - 5.0 * (t - 0.1)) ** 2 + (y - 2.0 * (t - 0.1)) ** 2) / (4 * t))

    rho = exact(0.1)
    Q = np.stack([rho, 5 * rho, 0 * rho, 2 * rho])[:, None]
    ones = np.ones((N, N))
    tr = T.Transport(g, ones, nu=ones, Sc=np.ones(1), bc=(T.OUTFLOW,) * 4)
    gpu = coag_mod.DustTransport(R_e, th_e, 1, ones, nu=ones, Sc=np.ones(1), geometry="cartesian",
                                 bc=(T.OUTFLOW,) * 4)
    q = torch.as_tensor(Q, device="cuda").contiguous()
    torch.cuda.synchronize()
    t = 0.1
    while t < 1.0 - 1e-12:
        dt = min(tr.cfl_dt(Q), 1.0 - t)
        Q = tr.step(Q, dt)
        gpu.step(q, dt)
        t += dt
    torch.cuda.synchronize()
    got = q.cpu().numpy()
    compare(got, Q, tol=1e-10)
    e_gpu = math.sqrt(np.mean((got[0, 0] - exact(1.0)) ** 2))
    e_ora = math.sqrt(np.mean((Q[0, 0] - exact(1.0)) ** 2))
    assert abs(e_gpu - e_ora) <= 1e-8 * e_ora


def test_bench_grid_transport_matches_oracle(coag_mod):
    """128 R x 64 theta cells x 100 species (the coagulation bench grid with
    its bins as the dust species), paper boundaries, diffusion, no sources
    (the oracle's source update is a per-cell loop): one step of every cell
    and species against the oracle."""
    nR, nZ, ns = 128, 64, 100
    R_e, th_e, Q, rho_g, nu, Sc, src = disc_setup(nR, nZ, ns, seed=11, R0=5.0, R1=100.0)
    g = T.Grid(R_e, th_e)
    tr = T.Transport(g, rho_g, nu=nu, Sc=Sc, bc=BCS["paper"])
    dt = 0.5 * tr.cfl_dt(Q)
    want = tr.step(Q, dt)
    gpu = coag_mod.DustTransport(R_e, th_e, ns, rho_g, nu=nu, Sc=Sc, bc=BCS["paper"])
    q = torch.as_tensor(Q, device="cuda").contiguous()
    torch.cuda.synchronize()
    gpu.step(q, dt)
    torch.cuda.synchronize()
    compare(q.cpu().numpy(), want)
    gpu.close()


def test_bench_grid_with_sources_conserves_mass(coag_mod):
    """The same grid with sources and closed boundaries: 10 steps keep every
    species' total mass to 1e-13 (a property at any size; the sources do not
    change densities)."""
    nR, nZ, ns = 128, 64, 100
    R_e, th_e, Q, rho_g, nu, Sc, src = disc_setup(nR, nZ, ns, seed=12, R0=5.0, R1=100.0)
    gpu = coag_mod.DustTransport(R_e, th_e, ns, rho_g, nu=nu, Sc=Sc, bc=BCS["closed"], sources=src)
    V = gpu.geometry()[0]
    q = torch.as_tensor(Q, device="cuda").contiguous()
    m0 = (q[0] * V[None]).sum(dim=(1, 2))
    g = T.Grid(R_e, th_e)
    dt = min(0.3 * T.Transport(g, rho_g, nu=nu, Sc=Sc).cfl_dt(Q), 0.02 / math.sqrt(G_M / R_e[0] ** 3))
    for _ in range(10):
        gpu.step(q, dt)
    m1 = (q[0] * V[None]).sum(dim=(1, 2))
    assert torch.all(torch.abs(m1 / m0 - 1) < 1e-13), (m1 / m0 - 1).abs().max().item()
    assert torch.isfinite(q).all()
    gpu.close()


def test_update_gas_matches_a_fresh_context(coag_mod):
    """Changing rho_g, nu and Sc in place, then cudisc_dust_update_gas, gives
    the step of a context built on the new gas, bitwise (the stencil and the
    cached reciprocals of rho_g and Sc are rebuilt)."""
    nR, nZ, ns = 21, 17, 4
    R_e, th_e, Q, rho_g, nu, Sc, src = disc_setup(nR, nZ, ns, seed=41)
    rng = np.random.default_rng(42)
    rho_g2, nu2, Sc2 = rho_g * (1 + 0.2 * rng.random(rho_g.shape)), nu * 1.7, Sc * 0.8
    a = coag_mod.DustTransport(R_e, th_e, ns, rho_g, nu=nu, Sc=Sc, bc=BCS["paper"])
    b = coag_mod.DustTransport(R_e, th_e, ns, rho_g2, nu=nu2, Sc=Sc2, bc=BCS["paper"])
    dt = 0.3 * T.Transport(T.Grid(R_e, th_e), rho_g2, nu=nu2, Sc=Sc2).cfl_dt(Q)
    a.gas("rho_g").copy_(torch.as_tensor(rho_g2))
    a.gas("nu").copy_(torch.as_tensor(nu2))
    a.gas("Sc").copy_(torch.as_tensor(Sc2))
    a.update_gas()
    qa = torch.as_tensor(Q, device="cuda").contiguous()
    qb = qa.clone()
    for _ in range(2):
        a.step(qa, dt)
        b.step(qb, dt)
    torch.cuda.synchronize()
    assert torch.equal(qa, qb)
    a.close()
    b.close()


@pytest.mark.parametrize("shape", [(1, 1), (1, 6), (6, 1), (2, 2)])
@pytest.mark.parametrize("bc", list(BCS))
def test_degenerate_grids_match_oracle(coag_mod, shape, bc):
    """One or two cells along a direction: every face is a boundary face or
    borders a ghost cell, and the stencil partners are ghosts.  Diffusion and
    sources on, two steps against the oracle."""
    nR, nZ = shape
    ns = 2
    R_e, th_e, Q, rho_g, nu, Sc, src = disc_setup(nR, nZ, ns, seed=5 + nR + 7 * nZ, R0=5.0, R1=6.0)
    g = T.Grid(R_e, th_e)
    tr = T.Transport(g, rho_g, nu=nu, Sc=Sc, bc=BCS[bc], floor=1e-25, sources=src)
    gpu = coag_mod.DustTransport(R_e, th_e, ns, rho_g, nu=nu, Sc=Sc, bc=BCS[bc], floor=1e-25, sources=src)
    q = torch.as_tensor(Q, device="cuda").contiguous()
    want = Q
    for _ in range(2):
        dt = min(0.5 * tr.cfl_dt(want), 0.02 / math.sqrt(G_M / R_e[0] ** 3))
        want = tr.step(want, dt)
        gpu.step(q, dt)
    torch.cuda.synchronize()
    compare(q.cpu().numpy(), want)
    gpu.close()
