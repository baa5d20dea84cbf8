"""Seeded synthetic disc inputs for the coagulation step.

This module builds INPUTS only: mass grids, gas fields of a smooth
protoplanetary disc on an (R, Z) grid, and initial dust densities.  It holds
none of the coagulation method's arithmetic (no collision kernel, no
relative velocities, no Stokes numbers, no mapping coefficients); both the
CUDA path and the CPU oracle consume what it returns.

Disc model (a stand-in for the gas structure the paper's dynamical, gas and
temperature solvers would supply; Sec. 7 of the paper lists the parameter
style used here):

* T(R) = T0 (R / 10 au)^-1/2, Sigma_g(R) = Sigma0 (R / 10 au)^-1,
  H/R = h0 (R / 10 au)^1/4,
* rho_g(R, Z) = Sigma_g / (sqrt(2 pi) H) exp(-Z^2 / 2 H^2), Z cell centres
  linear over 0..4H,
* eta(R) = (11/8) (H/R)^2, the midplane pressure-gradient parameter of this
  power-law disc (d ln P / d ln R = -11/4), used for the drift terms,
* initial dust: MRN, mass per logarithmic bin proportional to a^0.5 for
  a <= 1 micron and zero above, normalised to a dust-to-gas ratio of 0.01 in
  every cell (well mixed).

Size edges are log-spaced from a_min to a_max (N bins), edge masses are
m^e = 4/3 pi rho_m a_e^3 and bin-centre masses are the geometric midpoints of
neighbouring edges.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# CGS physical constants shared by both sides through the parameter struct.
CONST = dict(
    k_B=1.380649e-16,      # erg / K
    m_H=1.6735575e-24,     # g
    G=6.67430e-8,          # cm^3 g^-1 s^-2
    M_sun=1.98847e33,      # g
    au=1.495978707e13,     # cm
    yr=3.15576e7,          # s
    sigma_H2=2.0e-15,      # cm^2, H2 collision cross-section for nu_mol
)

KERNEL_PHYSICAL, KERNEL_CONSTANT, KERNEL_ADDITIVE = 0, 1, 2
FRAG_PHYSICAL, FRAG_NONE, FRAG_ALL = 0, 1, 2
SPLIT_MASS, SPLIT_NUMBER = 0, 1


def log_mass_grid(n_bins: int, a_min: float, a_max: float, rho_m: float):
    """N logarithmic bins whose outer size edges are a_min and a_max.

    Edge sizes are log-spaced (N+1 of them), edge masses m^e = 4/3 pi rho_m
    a_e^3, and centre masses are geometric midpoints of neighbouring edges.
    This reading reproduces the paper's m_{n+1}/m_n = 1.38 for both of its
    grids (Sec. 7: 100 bins over 0.1 um-0.5 cm and 135 over 0.1 um-20 cm);
    taking a_min and a_max as the outermost centres instead gives 1.39 for
    the first.
    """
    a_e = np.exp(np.linspace(np.log(a_min), np.log(a_max), n_bins + 1))
    me = 4.0 / 3.0 * np.pi * rho_m * a_e ** 3
    m = np.sqrt(me[:-1] * me[1:])
    a = np.sqrt(a_e[:-1] * a_e[1:])
    return m, me, a


def linear_mass_grid(n_bins: int, m0: float):
    """m_k = (k+1) m0 with edges at half-integers (for closed-form kernel tests)."""
    m = m0 * np.arange(1, n_bins + 1, dtype=np.float64)
    me = m0 * (np.arange(0, n_bins + 1, dtype=np.float64) + 0.5)
    return m, me


@dataclass
class Disc:
    """One coagulation problem: a grid of independent cells and a mass grid."""
    name: str
    n_R: int
    n_Z: int
    m: np.ndarray            # [N] bin-centre masses (g)
    me: np.ndarray           # [N+1] bin edges (g)
    rho_gas: np.ndarray      # [n_cells] g cm^-3
    T: np.ndarray            # [n_cells] K
    alpha: np.ndarray        # [n_cells]
    R: np.ndarray            # [n_cells] cm
    Z: np.ndarray            # [n_cells] cm
    eta: np.ndarray          # [n_cells] drift parameter
    rho0: np.ndarray         # [n_cells, N] initial dust densities
    t_span: float            # s
    v_frag: float = 100.0
    eta_frag: float = 11.0 / 6.0
    chi_im: float = 1.0
    rho_m: float = 1.6
    mu: float = 2.4
    Mstar: float = CONST["M_sun"]
    kernel_mode: int = KERNEL_PHYSICAL
    kernel_const: float = 0.0
    frag_mode: int = FRAG_PHYSICAL
    split_mode: int = SPLIT_MASS
    rtol: float = 1e-2
    atol_rel: float = 1e-10
    max_substeps: int = 2_000_000
    v_dust: np.ndarray | None = None   # [3, n_cells, N] or None
    vertical: int = 0                  # 1: surface densities, vertically integrated kernel
    R_edges: np.ndarray | None = None  # [n_R+1] cm, for cell volumes
    Z_edges: np.ndarray | None = None  # [n_R, n_Z+1] cm
    extra: dict = field(default_factory=dict)

    @property
    def n_cells(self) -> int:
        return self.rho_gas.shape[0]

    @property
    def n_bins(self) -> int:
        return self.m.shape[0]

    def scalars(self) -> dict:
        d = dict(v_frag=self.v_frag, eta_frag=self.eta_frag, chi_im=self.chi_im,
                 rho_m=self.rho_m, mu=self.mu, Mstar=self.Mstar,
                 k_B=CONST["k_B"], m_H=CONST["m_H"], G=CONST["G"],
                 sigma_H2=CONST["sigma_H2"], kernel_mode=self.kernel_mode,
                 kernel_const=self.kernel_const, frag_mode=self.frag_mode,
                 split_mode=self.split_mode, rtol=self.rtol,
                 atol_rel=self.atol_rel, max_substeps=self.max_substeps,
                 vertical=self.vertical)
        return d

    def subset(self, cells) -> "Disc":
        """The same problem restricted to a list of cells (cells are independent)."""
        cells = np.asarray(cells)
        kw = {k: getattr(self, k) for k in self.__dataclass_fields__}
        for k in ("rho_gas", "T", "alpha", "R", "Z", "eta"):
            kw[k] = np.ascontiguousarray(getattr(self, k)[cells])
        kw["rho0"] = np.ascontiguousarray(self.rho0[cells])
        if self.v_dust is not None:
            kw["v_dust"] = np.ascontiguousarray(self.v_dust[:, cells])
        kw["name"] = f"{self.name}[{len(cells)} cells]"
        kw["n_R"], kw["n_Z"] = len(cells), 1
        kw["R_edges"], kw["Z_edges"] = None, None
        kw["extra"] = dict(self.extra)
        return Disc(**kw)


def _disc_fields(R_c, n_Z, T0, Sigma0, h0, rng, rho_pert):
    au = CONST["au"]
    x = R_c / (10.0 * au)
    T_R = T0 * x ** -0.5
    Sig = Sigma0 * x ** -1.0
    hR = h0 * x ** 0.25
    H = hR * R_c
    # Z cell edges linear over 0..4H; centres at midpoints.
    fz = np.linspace(0.0, 4.0, n_Z + 1)
    Z_edges = H[:, None] * fz[None, :]
    Z_c = 0.5 * (Z_edges[:, 1:] + Z_edges[:, :-1])
    rho = Sig[:, None] / (np.sqrt(2 * np.pi) * H[:, None]) * np.exp(-0.5 * (Z_c / H[:, None]) ** 2)
    if rho_pert:
        rho = rho * np.exp(np.log(1.0 + rho_pert) * rng.standard_normal(rho.shape))
    T = np.repeat(T_R[:, None], n_Z, axis=1)
    Rg = np.repeat(R_c[:, None], n_Z, axis=1)
    eta = np.repeat((11.0 / 8.0 * hR ** 2)[:, None], n_Z, axis=1)
    return (rho.reshape(-1), T.reshape(-1), Rg.reshape(-1), Z_c.reshape(-1),
            eta.reshape(-1), Z_edges, Sig)


def mrn_initial(a, rho_gas, a_cut=1e-4, d2g=0.01):
    """MRN start: mass per log bin ~ a^0.5 up to a_cut, dust-to-gas d2g.  A
    grid whose smallest bin already lies above a_cut starts with all the
    dust in bin 0."""
    w = np.where(a <= a_cut * (1 + 1e-12), a ** 0.5, 0.0)
    if not w.sum() > 0.0:
        w = np.zeros_like(a, dtype=np.float64)
        w[0] = 1.0
    w = w / w.sum()
    return np.ascontiguousarray(d2g * rho_gas[:, None] * w[None, :])


def make_disc(n_R, n_Z, n_bins, a_min, a_max, R_in_au, R_out_au, t_span_yr,
              alpha=1e-3, v_frag=100.0, seed=None, rho_pert=0.0,
              alpha_dex=0.0, name="disc", T0=50.0, Sigma0=20.0, h0=0.05,
              rho_m=1.6):
    au, yr = CONST["au"], CONST["yr"]
    rng = np.random.default_rng(seed if seed is not None else 0)
    if n_R == 1:
        R_c = np.array([R_in_au * au])
        R_edges = np.array([R_in_au * au * 0.95, R_in_au * au * 1.05])
    else:
        R_edges = au * np.exp(np.linspace(np.log(R_in_au), np.log(R_out_au), n_R + 1))
        R_c = np.sqrt(R_edges[1:] * R_edges[:-1])
    rho, T, R, Z, eta, Z_edges, Sig = _disc_fields(R_c, n_Z, T0, Sigma0, h0, rng, rho_pert)
    n_cells = rho.shape[0]
    if alpha_dex:
        al = alpha * 10.0 ** (alpha_dex * rng.standard_normal(n_cells))
    else:
        al = np.full(n_cells, alpha)
    m, me, a = log_mass_grid(n_bins, a_min, a_max, rho_m)
    rho0 = mrn_initial(a, rho)
    return Disc(name=name, n_R=n_R, n_Z=n_Z, m=m, me=me, rho_gas=rho, T=T,
                alpha=al, R=R, Z=Z, eta=eta, rho0=rho0, t_span=t_span_yr * yr,
                v_frag=v_frag, rho_m=rho_m, R_edges=R_edges, Z_edges=Z_edges,
                extra=dict(a=a, Sigma_g=Sig))


# ---------------------------------------------------------------------------
# The five workloads: a single column, the 2D grid the throughput metric is
# quoted on, the adjoint problem, the large grid and a batch of uneven discs.
# ---------------------------------------------------------------------------

def column_1x32(seed=None, **kw) -> Disc:
    """1 R (10 au) x 32 Z, 50 bins 0.1 um - 1 cm, alpha 1e-3, v_frag 1 m/s, 1000 yr."""
    return make_disc(1, 32, 50, 1e-5, 1.0, 10.0, 10.0, 1000.0, alpha=1e-3,
                     v_frag=100.0, seed=seed, name="column_1x32_N50", **kw)


def grid_128x64(seed=1, **kw) -> Disc:
    """128 R (log 5-100 au) x 64 Z, 100 bins 0.1 um - 10 cm, 1e4 yr, +-10% rho_g."""
    return make_disc(128, 64, 100, 1e-5, 10.0, 5.0, 100.0, 1e4, alpha=1e-3,
                     v_frag=100.0, seed=seed, rho_pert=0.1, name="grid_128x64_N100", **kw)


def adjoint_64x32(v_frag=100.0, seed=2, **kw) -> Disc:
    """64 R x 32 Z, 80 bins 0.1 um - 1 cm, alpha lognormal 0.3 dex, 2000 yr."""
    return make_disc(64, 32, 80, 1e-5, 1.0, 5.0, 100.0, 2000.0, alpha=1e-3,
                     v_frag=v_frag, seed=seed, alpha_dex=0.3, name="adjoint_64x32_N80", **kw)


def grid_512x256(seed=3, **kw) -> Disc:
    """512 R x 256 Z, 150 bins 0.1 um - 100 cm, alpha 1e-4, v_frag 10 m/s, 1e4 yr."""
    return make_disc(512, 256, 150, 1e-5, 100.0, 5.0, 100.0, 1e4, alpha=1e-4,
                     v_frag=1000.0, seed=seed, name="grid_512x256_N150", **kw)


def batch_32_discs(seed=4):
    """32 independent discs with uneven cell and bin counts (log-uniform alpha)."""
    rng = np.random.default_rng(seed)
    discs = []
    for d in range(32):
        n_R = int(rng.integers(16, 257))
        n_Z = int(rng.integers(16, 129))
        n_b = int(rng.integers(40, 151))
        al = float(10.0 ** rng.uniform(-4, -2))
        vf = float(rng.uniform(100.0, 1000.0))
        discs.append(make_disc(n_R, n_Z, n_b, 1e-5, 10.0, 5.0, 100.0, 1e4,
                               alpha=al, v_frag=vf, seed=1000 + d,
                               name=f"batch{d}_{n_R}x{n_Z}_N{n_b}"))
    return discs


def make_ring_disc(n_R, n_bins, a_min, a_max, R_in_au, R_out_au, t_span_yr, alpha=1e-3,
                   v_frag=100.0, T=None, Sigma_g=None, mu=2.4, rho_m=1.6, d2g=0.01,
                   name="rings", seed=None):
    """Radii of a 1D disc for the vertically integrated kernel: the state is
    the dust SURFACE density per bin, rho_gas the mid-plane gas density
    Sigma_g / (sqrt(2 pi) H) with H = c_s / Omega_K of an isothermal column
    (gas structure, input only), Z = 0.

    T(R) = 36 K (R / 20 au)^-1/2 and Sigma_g = 10 g cm^-2 (R / 20 au)^-1 by
    default, so that the 20 au ring has the temperature of the paper's
    comparison with a surface-density code (Sec. 5.1: 20 au, 36 K, mu 2.4,
    alpha 1e-3, v_frag 1 m/s); the surface density is not given there and
    is a choice of this generator.  Initial dust: MRN below 1 micron with
    dust-to-gas ratio d2g (in surface density)."""
    au, yr = CONST["au"], CONST["yr"]
    if n_R == 1:
        R = np.array([R_in_au * au])
    else:
        R_edges = au * np.exp(np.linspace(np.log(R_in_au), np.log(R_out_au), n_R + 1))
        R = np.sqrt(R_edges[1:] * R_edges[:-1])
    x = R / (20.0 * au)
    Tc = np.full(n_R, 36.0) * x ** -0.5 if T is None else np.broadcast_to(np.asarray(T, float), (n_R,)).copy()
    Sg = 10.0 * x ** -1.0 if Sigma_g is None else np.broadcast_to(np.asarray(Sigma_g, float), (n_R,)).copy()
    cs = np.sqrt(CONST["k_B"] * Tc / (mu * CONST["m_H"]))
    Om = np.sqrt(CONST["G"] * CONST["M_sun"] / R ** 3)
    H = cs / Om
    rho_mid = Sg / (np.sqrt(2 * np.pi) * H)
    m, me, a = log_mass_grid(n_bins, a_min, a_max, rho_m)
    rng = np.random.default_rng(seed if seed is not None else 0)
    al = np.full(n_R, alpha) if seed is None else alpha * 10.0 ** (0.2 * rng.standard_normal(n_R))
    sig0 = mrn_initial(a, Sg, d2g=d2g)
    return Disc(name=name, n_R=n_R, n_Z=1, m=m, me=me, rho_gas=rho_mid, T=Tc, alpha=al, R=R,
                Z=np.zeros(n_R), eta=11.0 / 8.0 * (H / R) ** 2, rho0=sig0, t_span=t_span_yr * yr,
                v_frag=v_frag, rho_m=rho_m, mu=mu, vertical=1, extra=dict(a=a, H=H, Sigma_g=Sg))


def ring_20au(**kw) -> Disc:
    """One ring at 20 au with the paper's comparison parameters (Sec. 5.1),
    150 bins 0.1 um - 10 cm (the paper used 200 species; 160 is this
    library's limit), 1e4 yr."""
    return make_ring_disc(1, 150, 1e-5, 10.0, 20.0, 20.0, 1e4, alpha=1e-3, v_frag=100.0,
                          name="ring_20au_N150", **kw)


def rings_4096(seed=8, **kw) -> Disc:
    """4096 rings log-spaced over 5-100 au, 100 bins 0.1 um - 10 cm,
    alpha 1e-3 (0.2 dex scatter), v_frag 1 m/s, 1e4 yr."""
    return make_ring_disc(4096, 100, 1e-5, 10.0, 5.0, 100.0, 1e4, alpha=1e-3, v_frag=100.0,
                          seed=seed, name="rings_4096_N100", **kw)


def hse_inputs(disc: Disc, t_rise=0.0):
    """Inputs of the hydrostatic-equilibrium gas density for the (R, Z) grid
    of a disc from make_disc: cell centres R, Z and temperatures T as
    [n_R, n_Z] arrays, cylindrical cell volumes per radian V = (R dR) dZ
    with (R dR) = (R_{i+1}^2 - R_i^2) / 2 over the radial edges, those edges,
    and the column surface densities.  The grid holds the upper half of each
    column (Z >= 0), so its surface density is half of Sigma_g.  t_rise > 0
    warms the upper layers: T = T_mid (1 + t_rise (Z / Z_top)^2), Z_top the
    column's upper edge (a stand-in for a temperature solver's output)."""
    n_R, n_Z = disc.n_R, disc.n_Z
    R = disc.R.reshape(n_R, n_Z)
    Z = disc.Z.reshape(n_R, n_Z)
    Ze = disc.Z_edges
    T = disc.T.reshape(n_R, n_Z) * (1.0 + t_rise * (Z / Ze[:, -1:]) ** 2)
    RdR = 0.5 * (disc.R_edges[1:] ** 2 - disc.R_edges[:-1] ** 2)
    V = RdR[:, None] * np.diff(Ze, axis=1)
    return dict(R=np.ascontiguousarray(R), Z=np.ascontiguousarray(Z), T=np.ascontiguousarray(T),
                V=np.ascontiguousarray(V), R_edges=np.ascontiguousarray(disc.R_edges),
                Sigma_g=np.ascontiguousarray(0.5 * disc.extra["Sigma_g"]), mu=disc.mu,
                m_H=CONST["m_H"], k_B=CONST["k_B"], GM=CONST["G"] * disc.Mstar)


def adjoint_loss_weights(disc: Disc, a_max_small=1e-3):
    """Weights w[c,k] so that L = sum w * rho(T) is the mass of grains below
    10 um above Z = 1 H: cell volume V = 1/3 d(R^3) d(tan theta) for cells
    with Z > H, bins with a_k < 10 um."""
    a = disc.extra["a"]
    Re = disc.R_edges
    Ze = disc.Z_edges
    R_c = np.sqrt(Re[1:] * Re[:-1])
    tan_e = Ze / R_c[:, None]
    dR3 = (Re[1:] ** 3 - Re[:-1] ** 3)[:, None]
    V = dR3 / 3.0 * (tan_e[:, 1:] - tan_e[:, :-1])
    H = Ze[:, -1] / 4.0
    Zc = 0.5 * (Ze[:, 1:] + Ze[:, :-1])
    mask = (Zc > H[:, None]).astype(np.float64)
    w_cell = (V * mask).reshape(-1)
    w_bin = (a < a_max_small).astype(np.float64)
    return np.ascontiguousarray(w_cell[:, None] * w_bin[None, :])


def random_state(disc: Disc, seed=0, spread=6.0):
    """A seeded dense dust state (all bins populated) for RHS parity checks:
    per-bin densities log-uniform over `spread` decades, scaled to 1% of rho_g."""
    rng = np.random.default_rng(seed)
    x = 10.0 ** (-spread * rng.random((disc.n_cells, disc.n_bins)))
    x = x / x.sum(axis=1, keepdims=True)
    return np.ascontiguousarray(0.01 * disc.rho_gas[:, None] * x)


def transport_disc(n_R=128, n_Z=64, n_species=100, seed=21, R_in_au=5.0, R_out_au=100.0, th_max=0.25):
    """Inputs of the dust transport step (Sec. 3.1) on an (R, theta) grid:
    log-spaced radial edges, polar-angle edges 0..th_max above the mid-plane,
    a Gaussian gas disc (T-derived c_s, alpha = 1e-3 viscosity), dust species
    of sizes 1 um - 1 cm at 1 % of the gas with near-Keplerian velocities,
    Schmidt numbers 1, and the source-update fields (c_s, v_g, a, rho_m, GM).
    Returns a dict of host arrays; Q is [4, n_species, n_R, n_Z]."""
    au, G, Ms = CONST["au"], CONST["G"], CONST["M_sun"]
    rng = np.random.default_rng(seed)
    R_e = au * np.geomspace(R_in_au, R_out_au, n_R + 1)
    th_e = np.linspace(0.0, th_max, n_Z + 1)
    Rc = 0.5 * (R_e[1:] + R_e[:-1])
    thc = 0.5 * (th_e[1:] + th_e[:-1])
    Z = Rc[:, None] * np.tan(thc)[None, :]
    GM = G * Ms
    cs = 1e5 * (Rc / au / 10.0) ** -0.25
    Om = np.sqrt(GM / Rc ** 3)
    H = cs / Om
    rho_g = 1e-10 * ((Rc / au) ** -2.25)[:, None] * np.exp(-0.5 * (Z / H[:, None]) ** 2)
    nu = 1e-3 * (cs * H)[:, None] * np.ones((1, n_Z))
    vK = np.sqrt(GM / Rc)
    a = np.geomspace(1e-4, 1.0, n_species)
    P = np.zeros((4, n_species, n_R, n_Z))
    P[0] = 0.01 / n_species * rho_g[None] * (1 + 0.1 * rng.random((n_species, n_R, n_Z)))
    P[1] = -30.0 * rng.random((n_species, n_R, n_Z))
    P[2] = vK[None, :, None] * (1 + 1e-3 * rng.normal(size=(n_species, n_R, n_Z)))
    P[3] = -Z[None] * Om[None, :, None] * 1e-2 * rng.random((n_species, n_R, n_Z))
    Q = np.stack([P[0], P[0] * P[1], P[0] * P[2] * Rc[None, :, None], P[0] * P[3]])
    return dict(R_e=R_e, th_e=th_e, Q=np.ascontiguousarray(Q), rho_g=rho_g, nu=nu, Sc=np.ones(n_species),
                sources=dict(c_s=np.repeat(cs[:, None], n_Z, 1),
                             v_g=np.stack([0 * Z, vK[:, None] * np.ones((1, n_Z)), 0 * Z]),
                             a=a, rho_m=1.6, GM=GM),
                dt=0.02 / np.sqrt(GM / R_e[0] ** 3))
