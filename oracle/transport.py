"""transport.py -- plain FP64 CPU oracle of the dust transport step of Sec. 3.1
and 3.2 of Robinson, Booth & Owen, "Introducing cuDisc" (arXiv 2402.18471),
with the non-orthogonal diffusion stencil of Sec. 3.2 and Appendix A.

TEST INFRASTRUCTURE.  Only the tests and bench.py's CPU legs use it; it shares
no code with the CUDA library.

Grid (Sec. 2): cells (i, j), i along R (edges R^e_i), j along the polar angle
theta above the mid-plane (edges theta^e_j); cell centres (R^c_i, Z^c_ij =
R^c_i tan theta^c_j).  Volumes and face areas (Eqs. for V, A^R, A^Z):
  cylindrical:  V = d(R^3)/3 d(tan th),  A^R = (R^e)^2 d(tan th),  A^Z = d(R^2)/2 / cos th^e
  cartesian:    V = d(R^2)/2 d(tan th),  A^R = R^e d(tan th),      A^Z = dR / cos th^e
(the Cartesian form is the planar cell the paper's Gaussian-pulse test uses).
Radial faces have the unit normal (1, 0) in (R, Z); polar faces, the lines
Z = R tan th^e, have (-sin th^e, cos th^e).

Conserved quantities per species (Eq. quants): Q = (rho, rho v_R, rho v_phi R,
rho v_Z).  The full step (Sec. 3.1, items i-viii, following the VL2 scheme):
  (i)   first-order (donor cell) face states of the primitives at time n and
        the upwind advective flux of the pressureless Riemann problem (Eqs.
        roeav, riemann);
  (ii)  plus the diffusive flux at time n (Eqs. diffflux, Fdiffmom, fluxes);
  (iii) Q* = Q^n - dt/2 (FA)^n / V (Eqs. advdisc, fluxarea, halftimestepupdate);
  (iv)  the half-step source update (sources and implicit drag, dust.py);
  (v)   piecewise-linear face states of the n+1/2 primitives with the van Leer
        limiter generalised to non-uniform grids, and their advective flux;
  (vi)  plus the diffusive flux at n+1/2;
  (vii) Q^dag = Q^n - dt (FA)^(n+1/2) / V, then the full-step source update.
Ghost cells (two layers) are set before (i) and after (iv): outflow copies
the adjacent active cell, closed copies it and zeroes the flux through the
boundary face, zero sets the floor density at rest.

Readings (the paper is silent or inconsistent here; the CUDA path takes the
same ones):
  - primitives reconstructed: rho, v_R, the specific angular momentum
    l = v_phi R (= Q_2 / rho) and v_Z; a face state's conserved vector is
    (rho, rho v_R, rho l, rho v_Z);
  - the reconstruction coordinates are R along a row and tan(theta) along a
    column (the faces and centres of a column lie at R^c_i tan(theta));
  - generalised van Leer slope (after Mignone 2014) with forward and backward
    slopes s_F, s_B between centres and c_F = (xi_{i+1} - xi_i) / (x_{i+1/2}
    - xi_i), c_B = (xi_i - xi_{i-1}) / (xi_i - x_{i-1/2}):
      s = s_F s_B (c_F s_B + c_B s_F) / (s_B^2 + (c_F + c_B - 2) s_F s_B + s_F^2)
    when s_F s_B > 0, else 0 (the harmonic mean 2 s_F s_B / (s_F + s_B) on a
    uniform grid);
  - Riemann: the flux is 0 when v_l.n < 0 < v_r.n, else upwind by the sign
    of the Roe average (the mean of both sides when it is 0);
  - the diffusive momentum flux of Eq. Fdiffmom carries the transported
    component (v_R, l or v_Z) of the upwind face state of the diffusive mass
    flux, like the advective terms of Eq. dynfluxes;
  - the diffusion weights are w_k = (D_k / d_k) / (D_k / d_k + D_l / d_l):
    the printed mu = d / D is the inverse of what Eqs. F_k and vkl need for
    the flux of a piecewise-linear u with continuous normal flux to be exact;
  - stencil (Appendix A, the 3x3 block about a cell): across a radial face
    the cell on the low-R side pairs it with its lower polar face and the
    cell on the high-R side with its upper one ("clockwise"); across a polar
    face the lower cell pairs it with its inner radial face and the upper
    cell with its outer one ("anticlockwise");
  - the interpolation points lie on the faces' lines (orthogonal projections
    of the centres, not clamped to the segments);
  - ghost cells mirror the widths of the active cells next to the boundary;
    their gas density and viscosity copy the adjacent active cell.
Parity: pinned by tests/test_oracle_transport.py (limiter and Riemann cases,
the stencil's exact flux for linear and piecewise-linear fields on the
non-orthogonal grid, uniform states, mass conservation, and the second-order
convergence of the paper's advected-diffused Gaussian pulse, Sec. 3.4).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import dust

OUTFLOW, CLOSED, ZERO = 0, 1, 2
NG = 2                                   # ghost layers on every side


def vanleer_slope(sF, sB, cF, cB):
    """Generalised van Leer slope of a cell from its forward and backward
    slopes (per unit length) and the grid factors c_F, c_B."""
    sF = np.asarray(sF, dtype=np.float64)
    sB = np.asarray(sB, dtype=np.float64)
    num = sF * sB * (cF * sB + cB * sF)
    den = sB * sB + (cF + cB - 2.0) * sF * sB + sF * sF
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(sF * sB > 0.0, num / np.where(den == 0.0, 1.0, den), 0.0)
    return s


def riemann_flux(QL, QR, uL, uR, rhoL, rhoR):
    """Upwind advective flux of the pressureless Riemann problem (Eqs. roeav,
    riemann).  QL, QR: [4, ...] conserved face states; uL, uR: their normal
    velocities; rhoL, rhoR: their densities (>= 0)."""
    sl, sr = np.sqrt(np.maximum(rhoL, 0.0)), np.sqrt(np.maximum(rhoR, 0.0))
    den = sl + sr
    with np.errstate(invalid="ignore", divide="ignore"):
        vhat = np.where(den > 0.0, (sl * uL + sr * uR) / np.where(den > 0.0, den, 1.0), 0.0)
    FL, FR = QL * uL, QR * uR
    F = np.where(vhat > 0.0, FL, np.where(vhat < 0.0, FR, 0.5 * (FL + FR)))
    return np.where((uL < 0.0) & (uR > 0.0), 0.0, F)


class Grid:
    """The (R, theta) grid with two ghost layers on each side."""

    def __init__(self, R_e, th_e, R_c=None, th_c=None, geometry="cylindrical"):
        R_e = np.asarray(R_e, dtype=np.float64)
        th_e = np.asarray(th_e, dtype=np.float64)
        self.nR, self.nZ = R_e.size - 1, th_e.size - 1
        R_c = 0.5 * (R_e[1:] + R_e[:-1]) if R_c is None else np.asarray(R_c, dtype=np.float64)
        th_c = 0.5 * (th_e[1:] + th_e[:-1]) if th_c is None else np.asarray(th_c, dtype=np.float64)
        self.geometry = geometry
        self.Re = self._extend_edges(R_e)
        self.te_th = self._extend_edges(th_e)
        self.Rc = self._extend_centres(R_c, R_e)
        self.thc = self._extend_centres(th_c, th_e)
        if self.Re[0] <= 0.0:
            raise ValueError("ghost radii must stay positive")
        self.te = np.tan(self.te_th)              # tan theta at the edges
        self.tc = np.tan(self.thc)                # tan theta at the centres
        self.Zc = self.Rc[:, None] * self.tc[None, :]
        dR = np.diff(self.Re)
        dR2 = np.diff(self.Re ** 2)
        dR3 = np.diff(self.Re ** 3)
        dt = np.diff(self.te)
        if geometry == "cylindrical":
            self.V = dR3[:, None] / 3.0 * dt[None, :]
            self.AR = (self.Re ** 2)[:, None] * dt[None, :]                  # [nRg+1, nZg]
            self.AZ = (dR2 / 2.0)[:, None] / np.cos(self.te_th)[None, :]    # [nRg, nZg+1]
        elif geometry == "cartesian":
            self.V = dR2[:, None] / 2.0 * dt[None, :]
            self.AR = self.Re[:, None] * dt[None, :]
            self.AZ = dR[:, None] / np.cos(self.te_th)[None, :]
        else:
            raise ValueError(geometry)

    @staticmethod
    def _extend_edges(e):
        w = np.diff(e)
        lo = [e[0] - w[0], e[0] - w[0] - w[1 % w.size]]
        hi = [e[-1] + w[-1], e[-1] + w[-1] + w[-2 % w.size]]
        return np.concatenate([[lo[1], lo[0]], e, hi])

    @staticmethod
    def _extend_centres(c, e):
        # ghost centres mirror the active centres next to the boundary
        n = c.size
        lo = [2 * e[0] - c[0], 2 * e[0] - c[1 % n] if n > 1 else 2 * e[0] - c[0] - (e[1] - e[0])]
        hi = [2 * e[-1] - c[-1], 2 * e[-1] - c[-2] if n > 1 else 2 * e[-1] - c[-1] + (e[-1] - e[-2])]
        if n == 1:
            lo[1] = lo[0] - (e[1] - e[0])
            hi[1] = hi[0] + (e[1] - e[0])
        return np.concatenate([[lo[1], lo[0]], c, hi])

    @property
    def active(self):
        return (slice(NG, NG + self.nR), slice(NG, NG + self.nZ))

    def centre(self, i, j):
        return np.stack(np.broadcast_arrays(self.Rc[i], self.Rc[i] * self.tc[j]))


def fill_ghosts(Qa, bc, floor=0.0):
    """Active Q [4, ns, nR, nZ] -> ghosted [4, ns, nR+4, nZ+4]; bc = (inner
    R, outer R, lower theta, upper theta) boundary types.  The radial sides
    are set first, then the polar sides over whole columns (so the corners
    take the radial ghosts' values)."""
    f, ns, nR, nZ = Qa.shape
    Q = np.zeros((f, ns, nR + 2 * NG, nZ + 2 * NG))
    Q[:, :, NG:NG + nR, NG:NG + nZ] = Qa
    rest = np.zeros((4, 1, 1))
    rest[0] = floor
    for g in range(NG):
        for gi, si, kind in ((g, NG, bc[0]), (NG + nR + g, NG + nR - 1, bc[1])):
            Q[:, :, gi, NG:NG + nZ] = rest if kind == ZERO else Q[:, :, si, NG:NG + nZ]
    for g in range(NG):
        for gj, sj, kind in ((g, NG, bc[2]), (NG + nZ + g, NG + nZ - 1, bc[3])):
            Q[:, :, :, gj] = rest if kind == ZERO else Q[:, :, :, sj]
    return Q


def extend_cells(x, nR, nZ):
    """Per-cell array [nR, nZ] -> ghosted, copying the nearest active cell."""
    x = np.asarray(x, dtype=np.float64).reshape(nR, nZ)
    i = np.clip(np.arange(nR + 2 * NG) - NG, 0, nR - 1)
    j = np.clip(np.arange(nZ + 2 * NG) - NG, 0, nZ - 1)
    return x[i][:, j]


def primitives(Q):
    """rho, v_R, l = v_phi R, v_Z from Q (velocities 0 where rho <= 0)."""
    rho = Q[0]
    pos = rho > 0.0
    safe = np.where(pos, rho, 1.0)
    # divisions (not a reciprocal, which overflows for subnormal densities)
    return np.stack([rho, np.where(pos, Q[1] / safe, 0.0), np.where(pos, Q[2] / safe, 0.0),
                     np.where(pos, Q[3] / safe, 0.0)])


# ---- the diffusion stencil (Sec. 3.2, Appendix A) ---------------------------

def _face_line(grid, kind, i, j):
    """(point on the line, unit normal) of a face: kind 'R' = the radial face
    at R^e_i, kind 'Z' = the polar face at theta^e_j."""
    if kind == "R":
        return np.stack([grid.Re[i], 0.0 * grid.Re[i]]), np.array([1.0, 0.0])
    th = grid.te_th[j]
    return np.zeros(2), np.array([-math.sin(th), math.cos(th)])


def _proj(x, p0, n):
    """Orthogonal projection of point x onto the line through p0 with normal n."""
    return x - np.dot(x - p0, n) * n


def _interp_point(grid, D, kind, fi, fj, c1, c2):
    """Interpolation point on a face between cells c1 and c2: the weighted
    projections of their centres, weights w_c = (D_c/d_c) / sum over both."""
    p0, n = _face_line(grid, kind, fi, fj)
    x1, x2 = grid.centre(*c1), grid.centre(*c2)
    d1, d2 = abs(np.dot(x1 - p0, n)), abs(np.dot(x2 - p0, n))
    a1, a2 = D[c1] / d1, D[c2] / d2
    w1, w2 = a1 / (a1 + a2), a2 / (a1 + a2)
    return w1 * _proj(x1, p0, n) + w2 * _proj(x2, p0, n), w1, w2


def _solve2(v1, v2, n):
    det = v1[0] * v2[1] - v1[1] * v2[0]
    return (n[0] * v2[1] - n[1] * v2[0]) / det, (v1[0] * n[1] - v1[1] * n[0]) / det


def stencil_R(grid, D, i, j):
    """Coefficients of the net diffusive flux (per unit area, +R direction)
    through the radial face at R^e_{i+1} between k = (i, j) and l = (i+1, j)
    (ghosted indices): F = c_k u_k + c_l u_l + c_m u_m + c_p u_p, returned as
    [c_k, c_l, c_m, c_p].  Partner faces: below k (cells k, m = (i, j-1)) and
    above l (cells l, p = (i+1, j+1))."""
    k, l, m, p = (i, j), (i + 1, j), (i, j - 1), (i + 1, j + 1)
    y_s, wk, wl = _interp_point(grid, D, "R", i + 1, None, k, l)
    y_t, wk_t, wm = _interp_point(grid, D, "Z", None, j, k, m)          # face tau, below k
    y_n, wl_n, wp = _interp_point(grid, D, "Z", None, j + 1, l, p)      # face nu, above l
    xk, xl = grid.centre(*k), grid.centre(*l)
    n = np.array([1.0, 0.0])
    ckl, ckm = _solve2(y_s - xk, y_t - xk, n)
    clk, clp = _solve2(y_s - xl, y_n - xl, -n)
    # F_k = -D_k [w_l c_kl (u_l - u_k) + w_m c_km (u_m - u_k)], F_l likewise,
    # net = w_k F_k - w_l F_l; coefficients of u_k, u_l, u_m, u_p
    fk_l, fk_m = -D[k] * wl * ckl, -D[k] * wm * ckm
    fl_k, fl_p = -D[l] * wk * clk, -D[l] * wp * clp
    return np.array([wk * -(fk_l + fk_m) - wl * fl_k,
                     wk * fk_l - wl * -(fl_k + fl_p),
                     wk * fk_m,
                     -wl * fl_p])


def stencil_Z(grid, D, i, j):
    """The same for the polar face at theta^e_{j+1} between a = (i, j) and
    l = (i, j+1) (flux along its normal (-sin th, cos th)), returned as
    [c_a, c_l, c_m, c_b].  Partner faces: inside a (cells a, m = (i-1, j))
    and outside l (cells l, b = (i+1, j+1))."""
    a, l, m, b = (i, j), (i, j + 1), (i - 1, j), (i + 1, j + 1)
    y_l, wa, wl = _interp_point(grid, D, "Z", None, j + 1, a, l)
    y_b, wa_b, wm = _interp_point(grid, D, "R", i, None, a, m)          # face beta, inner side of a
    y_e, wl_e, wb = _interp_point(grid, D, "R", i + 1, None, l, b)      # face eps, outer side of l
    xa, xl = grid.centre(*a), grid.centre(*l)
    th = grid.te_th[j + 1]
    n = np.array([-math.sin(th), math.cos(th)])
    cal, cam = _solve2(y_l - xa, y_b - xa, n)
    cla, clb = _solve2(y_l - xl, y_e - xl, -n)
    # coefficients of u_a, u_l, u_m, u_b
    fa_l, fa_m = -D[a] * wl * cal, -D[a] * wm * cam
    fl_a, fl_b = -D[l] * wa * cla, -D[l] * wb * clb
    return np.array([wa * -(fa_l + fa_m) - wl * fl_a,
                     wa * fa_l - wl * -(fl_a + fl_b),
                     wa * fa_m,
                     -wl * fl_b])


def stencil_arrays(grid, D):
    """Coefficients of every active face's stencil: cR [4, nR+1, nZ] (radial
    faces, cells k, l, m, p) and cZ [4, nR, nZ+1] (polar faces, cells a, l,
    m, b).  D [nRg, nZg] per cell."""
    nR, nZ = grid.nR, grid.nZ
    cR = np.zeros((4, nR + 1, nZ))
    cZ = np.zeros((4, nR, nZ + 1))
    for a in range(nR + 1):
        for jj in range(nZ):
            cR[:, a, jj] = stencil_R(grid, D, NG - 1 + a, NG + jj)
    for ii in range(nR):
        for b in range(nZ + 1):
            cZ[:, ii, b] = stencil_Z(grid, D, NG + ii, NG - 1 + b)
    return cR, cZ


def diffusion_fluxes(grid, cR, cZ, u):
    """Net diffusive fluxes (per unit area, without 1/Sc) through the active
    radial faces [ns, nR+1, nZ] and polar faces [ns, nR, nZ+1] for the
    ghosted field u [ns, nRg, nZg]."""
    nR, nZ = grid.nR, grid.nZ
    k = u[:, NG - 1:NG + nR, NG:NG + nZ]
    l = u[:, NG:NG + nR + 1, NG:NG + nZ]
    m = u[:, NG - 1:NG + nR, NG - 1:NG + nZ - 1]
    p = u[:, NG:NG + nR + 1, NG + 1:NG + nZ + 1]
    FR = cR[0] * k + cR[1] * l + cR[2] * m + cR[3] * p
    a = u[:, NG:NG + nR, NG - 1:NG + nZ]
    l = u[:, NG:NG + nR, NG:NG + nZ + 1]
    m = u[:, NG - 1:NG + nR - 1, NG - 1:NG + nZ]
    b = u[:, NG + 1:NG + nR + 1, NG:NG + nZ + 1]
    FZ = cZ[0] * a + cZ[1] * l + cZ[2] * m + cZ[3] * b
    return FR, FZ


class Transport:
    """One dust transport step of Sec. 3.1 on a grid, for n_species fluids.

    rho_g, nu: [nR, nZ] gas density and viscosity (nu None: no diffusion);
    Sc: [n_species]; bc: four boundary types (inner R, outer R, lower theta,
    upper theta).  Sources (dict with c_s [nR, nZ], v_g [3, nR, nZ], a
    [n_species], rho_m, GM) or None: transport only."""

    def __init__(self, grid, rho_g, nu=None, Sc=None, bc=(OUTFLOW, OUTFLOW, CLOSED, OUTFLOW), floor=0.0,
                 sources=None):
        self.g = grid
        self.bc = tuple(bc)
        self.floor = floor
        nR, nZ = grid.nR, grid.nZ
        self.rho_g = extend_cells(rho_g, nR, nZ)
        self.nu = None if nu is None else extend_cells(nu, nR, nZ)
        self.Sc = None if Sc is None else np.asarray(Sc, dtype=np.float64)
        self.sources = sources
        if self.nu is not None:
            # the stencils of D = rho_g nu (the 1/Sc of each species scales them)
            self.cR, self.cZ = stencil_arrays(grid, self.rho_g * self.nu)

    # -- pieces ---------------------------------------------------------------
    def face_states(self, P, order):
        """Left and right primitive states at the radial faces [4, ns, nR+1,
        nZ] and at the polar faces [4, ns, nR, nZ+1]."""
        g = self.g
        nR, nZ = g.nR, g.nZ
        rows = np.arange(NG - 1, NG + nR + 1)      # cells either side of the active radial faces
        cols = np.arange(NG - 1, NG + nZ + 1)
        if order == 1:
            PL_R = P[:, :, NG - 1:NG + nR, NG:NG + nZ]
            PR_R = P[:, :, NG:NG + nR + 1, NG:NG + nZ]
            PL_Z = P[:, :, NG:NG + nR, NG - 1:NG + nZ]
            PR_Z = P[:, :, NG:NG + nR, NG:NG + nZ + 1]
            return PL_R, PR_R, PL_Z, PR_Z
        # slopes along R (coordinate R) of the cells NG-1 .. NG+nR
        x, e = g.Rc, g.Re
        i = rows
        sF = (P[:, :, i + 1, :] - P[:, :, i, :]) / (x[i + 1] - x[i])[None, None, :, None]
        sB = (P[:, :, i, :] - P[:, :, i - 1, :]) / (x[i] - x[i - 1])[None, None, :, None]
        cF = ((x[i + 1] - x[i]) / (e[i + 1] - x[i]))[None, None, :, None]
        cB = ((x[i] - x[i - 1]) / (x[i] - e[i]))[None, None, :, None]
        sR = vanleer_slope(sF, sB, cF, cB)        # [4, ns, nR+2, nZg]
        hiR = P[:, :, i, :] + sR * (e[i + 1] - x[i])[None, None, :, None]     # value at the cell's outer face
        loR = P[:, :, i, :] + sR * (e[i] - x[i])[None, None, :, None]         # at its inner face
        PL_R = hiR[:, :, :-1, NG:NG + nZ]
        PR_R = loR[:, :, 1:, NG:NG + nZ]
        # slopes along a column (coordinate tan theta)
        x, e = g.tc, g.te
        j = cols
        sF = (P[:, :, :, j + 1] - P[:, :, :, j]) / (x[j + 1] - x[j])
        sB = (P[:, :, :, j] - P[:, :, :, j - 1]) / (x[j] - x[j - 1])
        cF = (x[j + 1] - x[j]) / (e[j + 1] - x[j])
        cB = (x[j] - x[j - 1]) / (x[j] - e[j])
        sZ = vanleer_slope(sF, sB, cF, cB)
        hiZ = P[:, :, :, j] + sZ * (e[j + 1] - x[j])
        loZ = P[:, :, :, j] + sZ * (e[j] - x[j])
        PL_Z = hiZ[:, :, NG:NG + nR, :-1]
        PR_Z = loZ[:, :, NG:NG + nR, 1:]
        return PL_R, PR_R, PL_Z, PR_Z

    def fluxes(self, Qg, order):
        """Total fluxes (per unit area) through the active radial and polar faces."""
        g = self.g
        nR, nZ = g.nR, g.nZ
        P = primitives(Qg)
        PL_R, PR_R, PL_Z, PR_Z = self.face_states(P, order)

        def cons(Pf):
            return np.stack([Pf[0], Pf[0] * Pf[1], Pf[0] * Pf[2], Pf[0] * Pf[3]])

        # radial faces: normal (1, 0)
        FR = riemann_flux(cons(PL_R), cons(PR_R), PL_R[1], PR_R[1], PL_R[0], PR_R[0])
        # polar faces: normal (-sin th, cos th) at theta^e of the face
        th = g.te_th[NG:NG + nZ + 1][None, None, :]
        sn, cs = np.sin(th), np.cos(th)
        uL = -sn * PL_Z[1] + cs * PL_Z[3]
        uR = -sn * PR_Z[1] + cs * PR_Z[3]
        FZ = riemann_flux(cons(PL_Z), cons(PR_Z), uL, uR, PL_Z[0], PR_Z[0])
        if self.nu is not None:
            u = Qg[0] / self.rho_g[None]
            dR, dZ = diffusion_fluxes(g, self.cR, self.cZ, u)
            dR = dR / self.Sc[:, None, None]
            dZ = dZ / self.Sc[:, None, None]
            for F, d, PL, PR in ((FR, dR, PL_R, PR_R), (FZ, dZ, PL_Z, PR_Z)):
                up = np.where(d > 0.0, 1.0, 0.0)
                F[0] += d
                for f in (1, 2, 3):
                    F[f] += d * (up * PL[f] + (1.0 - up) * PR[f])
        # closed boundaries: no flux through the boundary faces
        if self.bc[0] == CLOSED:
            FR[:, :, 0, :] = 0.0
        if self.bc[1] == CLOSED:
            FR[:, :, -1, :] = 0.0
        if self.bc[2] == CLOSED:
            FZ[:, :, :, 0] = 0.0
        if self.bc[3] == CLOSED:
            FZ[:, :, :, -1] = 0.0
        return FR, FZ

    def flux_divergence(self, FR, FZ):
        """(FA) / V of every active cell (Eq. fluxarea)."""
        g = self.g
        nR, nZ = g.nR, g.nZ
        AR = g.AR[NG:NG + nR + 1, NG:NG + nZ]
        AZ = g.AZ[NG:NG + nR, NG:NG + nZ + 1]
        FA = (FR[:, :, 1:, :] * AR[1:, :] - FR[:, :, :-1, :] * AR[:-1, :] +
              FZ[:, :, :, 1:] * AZ[:, 1:] - FZ[:, :, :, :-1] * AZ[:, :-1])
        return FA / g.V[NG:NG + nR, NG:NG + nZ]

    def _sources(self, Q, Pact, h):
        """The source update of dust.py on active cells (Q, Pact [4, ns, nR, nZ];
        Pact with the azimuthal component as l = v_phi R)."""
        g = self.g
        nR, nZ = g.nR, g.nZ
        s = self.sources
        Rc = np.repeat(g.Rc[NG:NG + nR], nZ)
        Zc = g.Zc[NG:NG + nR, NG:NG + nZ].reshape(-1)
        ns = Q.shape[1]
        Pn = Pact.reshape(4, ns, -1).copy()
        Pn[2] = Pn[2] / Rc[None, :]
        out = dust.source_update(Q.reshape(4, ns, -1), Pn, h, Rc, Zc,
                                 self.rho_g[NG:NG + nR, NG:NG + nZ].reshape(-1),
                                 np.asarray(s["c_s"]).reshape(-1), np.asarray(s["v_g"]).reshape(3, -1),
                                 s["a"], s["rho_m"], s["GM"])
        return out.reshape(Q.shape)

    def step(self, Q, dt):
        """One full step: Q [4, ns, nR, nZ] (active cells) -> Q^{n+1}."""
        Q = np.asarray(Q, dtype=np.float64)
        g = self.g
        nR, nZ = g.nR, g.nZ
        Qg = fill_ghosts(Q, self.bc, self.floor)
        Pn = primitives(Q)
        FR, FZ = self.fluxes(Qg, order=1)
        Qh = Q - 0.5 * dt * self.flux_divergence(FR, FZ)
        if self.sources is not None:
            Qh = self._sources(Qh, Pn, 0.5 * dt)
        Ph = primitives(Qh)
        Qg = fill_ghosts(Qh, self.bc, self.floor)
        FR, FZ = self.fluxes(Qg, order=2)
        Qn = Q - dt * self.flux_divergence(FR, FZ)
        if self.sources is not None:
            Qn = self._sources(Qn, Ph, dt)
        return Qn

    def cfl_dt(self, Q, C_adv=0.4, C_diff=0.2):
        """The CFL step (Eqs. dtCFL, dt_adv, dt_diff) with dR, dZ the cell's
        radial width and the height of its column segment."""
        g = self.g
        nR, nZ = g.nR, g.nZ
        P = primitives(Q)
        dR = np.diff(g.Re)[NG:NG + nR][:, None] * np.ones((1, nZ))
        dZ = g.Rc[NG:NG + nR][:, None] * np.diff(g.te)[NG:NG + nZ][None, :]
        ns = Q.shape[1]
        nu = (self.nu[NG:NG + nR, NG:NG + nZ] if self.nu is not None else np.zeros((nR, nZ)))
        Sc = self.Sc if self.Sc is not None else np.ones(ns)
        return dust.cfl_dt(P[1].reshape(ns, -1), P[3].reshape(ns, -1), dR.reshape(-1), dZ.reshape(-1),
                           np.maximum(nu.reshape(-1), 1e-300), Sc, C_adv, C_diff)
