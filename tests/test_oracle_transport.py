"""Pins of the dust transport oracle (Sec. 3.1-3.2, Appendix A) against facts
that do not come from its code: the limiter's defining properties, the
pressureless Riemann problem's cases, the exact flux of the non-orthogonal
diffusion stencil for linear fields (and for a piecewise-linear field across
a jump of D, with continuous normal flux), the closed polygon of a planar
cell (a uniform state stays uniform), mass conservation with closed
boundaries, and the paper's own test: the second-order convergence of an
advected and diffused Gaussian pulse (Sec. 3.4, Eq. gaupulse)."""
import math

import numpy as np
import pytest

from oracle import transport as T


# ---- limiter ----------------------------------------------------------------

def test_limiter_uniform_grid_is_the_harmonic_mean():
    rng = np.random.default_rng(0)
    sF, sB = rng.uniform(0.1, 3, 50), rng.uniform(0.1, 3, 50)
    assert np.allclose(T.vanleer_slope(sF, sB, 2.0, 2.0), 2 * sF * sB / (sF + sB), rtol=1e-14)
    assert np.allclose(T.vanleer_slope(-sF, -sB, 2.0, 2.0), -2 * sF * sB / (sF + sB), rtol=1e-14)


def test_limiter_exact_for_linear_data_and_flat_at_extrema():
    rng = np.random.default_rng(1)
    s = rng.normal(size=40)
    cF, cB = rng.uniform(1.2, 3, 40), rng.uniform(1.2, 3, 40)
    assert np.allclose(T.vanleer_slope(s, s, cF, cB), s, rtol=1e-14)
    assert np.all(T.vanleer_slope(s, -s, cF, cB) == 0.0)
    assert np.all(T.vanleer_slope(s, 0 * s, cF, cB) == 0.0)


def test_limited_face_values_stay_between_the_neighbours():
    """On a non-uniform 1D grid with cell centres at the midpoints and
    neighbouring widths within 25 % of each other (c_F, c_B in [1.8, 2.25]),
    the face values q_i + s (x_face - xi_i) of monotone data lie between the
    neighbouring cell values.  (The bound needs c_F (c_B - 1) + c_B (c_B - 2)
    >= 0 and its mirror; a neighbour under half as wide breaks it.)"""
    rng = np.random.default_rng(2)
    for _ in range(400):
        w = np.cumprod(np.concatenate([[1.0], rng.uniform(0.8, 1.25, 2)]))
        e = np.concatenate([[0.0], np.cumsum(w)])
        x = 0.5 * (e[1:] + e[:-1])
        q = np.sort(rng.normal(size=3)) * rng.choice([-1, 1])
        sF = (q[2] - q[1]) / (x[2] - x[1])
        sB = (q[1] - q[0]) / (x[1] - x[0])
        cF = (x[2] - x[1]) / (e[2] - x[1])
        cB = (x[1] - x[0]) / (x[1] - e[1])
        s = float(T.vanleer_slope(sF, sB, cF, cB))
        hi, lo = q[1] + s * (e[2] - x[1]), q[1] + s * (e[1] - x[1])
        assert min(q[1], q[2]) - 1e-12 <= hi <= max(q[1], q[2]) + 1e-12
        assert min(q[0], q[1]) - 1e-12 <= lo <= max(q[0], q[1]) + 1e-12


# ---- Riemann problem of pressureless dust ----------------------------------

def Qof(rho, v):
    return np.array([rho, rho * v, rho * 2.0, rho * 0.5])


@pytest.mark.parametrize("rl,ul,rr,ur,want", [
    (1.0, 2.0, 3.0, 1.0, "L"),        # both move right: upwind is left
    (1.0, -1.0, 3.0, -2.0, "R"),      # both move left: upwind is right
    (4.0, 1.0, 1.0, -1.5, "L"),       # collision (delta shock): Roe average (2 - 1.5)/3 > 0 moves right
    (1.0, 1.0, 4.0, -1.5, "R"),       # collision, Roe average (1 - 3)/3 < 0 moves left
    (1.0, -1.0, 1.0, 2.0, "0"),       # diverging: vacuum at the face
    (4.0, 1.0, 1.0, -2.0, "M"),       # Roe average exactly 0: the mean of both fluxes
])
def test_riemann_cases(rl, ul, rr, ur, want):
    QL, QR = Qof(rl, ul), Qof(rr, ur)
    F = T.riemann_flux(QL, QR, np.float64(ul), np.float64(ur), np.float64(rl), np.float64(rr))
    expect = {"L": QL * ul, "R": QR * ur, "0": 0 * QL, "M": 0.5 * (QL * ul + QR * ur)}[want]
    assert np.allclose(F, expect, rtol=1e-15, atol=0)


# ---- the non-orthogonal diffusion stencil -----------------------------------

def grid(geometry, nR=6, nZ=5, th0=0.0, th1=0.6, seed=3):
    rng = np.random.default_rng(seed)
    Re = 10.0 * np.cumprod(np.concatenate([[1.0], rng.uniform(1.05, 1.3, nR)]))
    te = np.linspace(th0, th1, nZ + 1)
    return T.Grid(Re, te, geometry=geometry)


@pytest.mark.parametrize("geometry", ["cylindrical", "cartesian"])
def test_stencil_exact_for_a_linear_field(geometry):
    """u = a R + b Z + c with a constant D: every face's net flux is
    -D grad(u).n, although the grid is not orthogonal."""
    g = grid(geometry, th0=-0.3, th1=0.7)
    D = np.full((g.nR + 4, g.nZ + 4), 2.5)
    aa, bb = 0.7, -1.3
    u = (aa * g.Rc[:, None] + bb * g.Zc + 4.0)[None]
    cR, cZ = T.stencil_arrays(g, D)
    FR, FZ = T.diffusion_fluxes(g, cR, cZ, u)
    assert np.allclose(FR, -2.5 * aa, rtol=1e-11, atol=0)
    th = g.te_th[T.NG:T.NG + g.nZ + 1]
    want = -2.5 * (-np.sin(th) * aa + np.cos(th) * bb)
    assert np.allclose(FZ[0], np.broadcast_to(want, FZ[0].shape), rtol=1e-11, atol=1e-13)


def test_stencil_exact_across_a_jump_of_D():
    """D = D1 for R < R^e_3 and D2 beyond: u piecewise linear in R with
    D1 u'_1 = D2 u'_2 (continuous flux) plus a linear Z part; the radial
    faces carry exactly -D u'."""
    g = grid("cylindrical", nR=6, nZ=4, th0=0.0, th1=0.5, seed=4)
    Rj = g.Re[T.NG + 3]
    D1, D2, g1 = 1.0, 4.0, 0.8
    g2 = D1 * g1 / D2
    Rc = g.Rc[:, None]
    D = np.where(Rc < Rj, D1, D2) * np.ones_like(g.Zc)
    # piecewise linear in R, continuous at Rj; the Z part has the same gradient
    # on both sides, so D grad(u).n of the radial faces is D u'_R alone
    u = (np.where(Rc < Rj, g1 * (Rc - Rj), g2 * (Rc - Rj)) * np.ones_like(g.Zc))[None]
    cR, cZ = T.stencil_arrays(g, D)
    FR, _ = T.diffusion_fluxes(g, cR, cZ, u)
    assert np.allclose(FR[0], -D1 * g1, rtol=1e-11, atol=0)


# ---- whole steps ------------------------------------------------------------

def test_uniform_state_stays_uniform_on_planar_cells():
    """In the Cartesian geometry the faces of a cell close (sum of n A = 0),
    so a uniform density moving uniformly, with uniform diffusion, stays
    uniform under outflow boundaries."""
    g = grid("cartesian", nR=7, nZ=6, th0=-0.4, th1=0.5)
    ns = 2
    P = np.zeros((4, ns, g.nR, g.nZ))
    P[0] = 3.0
    P[1] = 0.7
    P[2] = 0.0
    P[3] = -0.4
    Q = np.stack([P[0], P[0] * P[1], P[0] * P[2], P[0] * P[3]])
    tr = T.Transport(g, np.ones((g.nR, g.nZ)), nu=np.ones((g.nR, g.nZ)), Sc=np.ones(ns),
                     bc=(T.OUTFLOW,) * 4)
    out = tr.step(Q, 0.05)
    assert np.allclose(out, Q, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("geometry", ["cylindrical", "cartesian"])
def test_mass_conserved_with_closed_boundaries(geometry):
    g = grid(geometry, nR=8, nZ=7, th0=0.0, th1=0.5, seed=6)
    rng = np.random.default_rng(7)
    ns = 3
    P = np.zeros((4, ns, g.nR, g.nZ))
    P[0] = rng.uniform(0.5, 2.0, P[0].shape)
    P[1] = rng.normal(0, 0.3, P[1].shape)
    P[2] = rng.normal(0, 0.3, P[2].shape)
    P[3] = rng.normal(0, 0.3, P[3].shape)
    Q = np.stack([P[0], P[0] * P[1], P[0] * P[2], P[0] * P[3]])
    rho_g = rng.uniform(0.5, 1.5, (g.nR, g.nZ))
    nu = rng.uniform(0.5, 1.5, (g.nR, g.nZ))
    tr = T.Transport(g, rho_g, nu=nu, Sc=np.array([1.0, 2.0, 0.5]), bc=(T.CLOSED,) * 4)
    V = g.V[T.NG:T.NG + g.nR, T.NG:T.NG + g.nZ]
    m0 = (Q[0] * V).sum(axis=(1, 2))
    dt = 0.3 * tr.cfl_dt(Q)
    for _ in range(5):
        Q = tr.step(Q, dt)
    m1 = (Q[0] * V).sum(axis=(1, 2))
    assert np.allclose(m1, m0, rtol=1e-13, atol=0)
    assert np.all(Q[0] > 0)


def gaussian_pulse_error(N, background=0.01):
    """The paper's test (Sec. 3.4): rho = A/t exp(-((x - x_p)^2 + (y - y_p)^2)
    / (4 D t)), A = D = 1, (x0, y0) = (30, 0), t0 = 0.1, (v_x, v_y) = (5, 2),
    from t0 to 1 on N x N cells, log-spaced in R over 10-50 and linear in
    theta over -pi/6..pi/6, Cartesian areas and volumes, outflow boundaries.
    A uniform background density is added (uniform advection and diffusion
    carry it unchanged, so the closed form is background + pulse): on the
    coarse grids the pulse at t0 (width 0.45) spans about one cell, and the
    undershoots of the limited scheme at its edge would otherwise take the
    far field's zero density below zero.  Returns the L2 norm of the error
    against the closed form at t = 1."""
    Re = np.geomspace(10.0, 50.0, N + 1)
    te = np.linspace(-math.pi / 6, math.pi / 6, N + 1)
    g = T.Grid(Re, te, geometry="cartesian")
    a = T.NG
    x = g.Rc[a:a + N][:, None] * np.ones((1, N))
    y = g.Zc[a:a + N, a:a + N]
    vx, vy, t0, t1 = 5.0, 2.0, 0.1, 1.0

    def exact(t):
        xp, yp = 30.0 + vx * (t - t0), 0.0 + vy * (t - t0)
        return background + 1.0 / t * np.exp(-((x - xp) ** 2 + (y - yp) ** 2) / (4.0 * t))

    rho = exact(t0)
    Q = np.stack([rho, rho * vx, 0 * rho, rho * vy])[:, None]
    tr = T.Transport(g, np.ones((N, N)), nu=np.ones((N, N)), Sc=np.ones(1), bc=(T.OUTFLOW,) * 4)
    t = t0
    while t < t1 - 1e-12:
        dt = min(tr.cfl_dt(Q), t1 - t)
        Q = tr.step(Q, dt)
        t += dt
    assert Q[0].min() > 0.0
    return math.sqrt(np.mean((Q[0, 0] - exact(t1)) ** 2))


def test_gaussian_pulse_converges_at_second_order():
    """L2 error proportional to 1/N^2 (the paper's Fig. l2error): the ratio
    between N = 48 and 96 is near 4 once the initial pulse is resolved."""
    e = [gaussian_pulse_error(N) for N in (24, 48, 96)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert r1 > 1.8 and r2 > 3.3, (e, r1, r2)
