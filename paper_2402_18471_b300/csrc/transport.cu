// The dust transport step of Sec. 3.1-3.2 on the (R, theta) grid of Sec. 2:
// per species a pressureless fluid, advanced by the two-stage (VL2) scheme
// the paper follows.  Stage 1 takes donor-cell face states, stage 2
// piecewise-linear ones with the van Leer limiter generalised to non-uniform
// grids; both take the upwind flux of the pressureless Riemann problem by the
// sign of the Roe-averaged normal velocity (Eqs. roeav, riemann) plus the
// turbulent diffusion flux of Eq. (diffflux) through the non-orthogonal
// stencil of Sec. 3.2 / Appendix A, and the momenta carry their upwind
// component (Eq. Fdiffmom).  Between and after the stages the source update
// of dust.cu (sources, implicit drag) runs when sources are given.
//
// Layout: Q [4][n_species][n_R n_Z] FP64, Q = (rho, rho v_R, rho v_phi R,
// rho v_Z), cell c = i n_Z + j (i along R, j along theta).  Workspace of the
// context: the ghosted primitives (two ghost layers a side) [4][n_s][(n_R +
// 4)(n_Z + 4)], the face fluxes of the radial faces [4][n_s][(n_R + 1) n_Z]
// and polar faces [4][n_s][n_R (n_Z + 1)], the half-step state, the
// start-of-stage primitives of the source update, the species-free stencil
// coefficients of every face (4 each), and per ghosted cell the limited
// slopes along R and theta [4][n_s][ng] and the diffusion variable u
// [n_s][ng].  FP64 throughout: the step is a handful of passes over Q,
// bound by FP64 issue and HBM.
//
// Readings of the paper (the same as the FP64 oracle's): the azimuthal
// primitive reconstructed is l = v_phi R; reconstruction coordinates are R
// along a row and tan(theta) along a column; the diffusion weights are
// w_k = (D_k / d_k) / (D_k / d_k + D_l / d_l); across a radial face the low-R
// cell pairs it with its lower polar face and the high-R cell with its upper
// one, across a polar face the lower cell with its inner radial face and the
// upper cell with its outer one; ghost cells mirror the boundary cells'
// widths and copy their gas; a density <= 0 has zero velocity.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "coag_internal.h"

struct cudisc_dust_ctx {
    cudisc_dust_params p;
    cudaStream_t stream = nullptr;
    int ns = 0, nR = 0, nZ = 0, nRg = 0, nZg = 0;
    std::string err;
    // geometry (ghosted where marked g)
    double *Rc = nullptr, *tc = nullptr;          // g: [nRg], [nZg]
    double *Re = nullptr, *te = nullptr;          // g: [nRg + 1], [nZg + 1] (te = tan theta^e)
    double *sn = nullptr, *cs = nullptr;          // g: sin, cos theta^e [nZg + 1]
    double *V = nullptr, *AR = nullptr, *AZ = nullptr;   // [nR nZ], [(nR + 1) nZ], [nR (nZ + 1)]
    double *Rcell = nullptr, *Zcell = nullptr;    // [nR nZ] cell centres (sources)
    double *iV = nullptr, *iRcell = nullptr;      // [nR nZ] 1 / V, 1 / R of the cell centres
    double *irg = nullptr, *iSc = nullptr;        // [nR nZ] 1 / rho_g, [n_s] 1 / Sc (with diffusion)
    double *cR = nullptr, *cZ = nullptr;          // [4][faces] stencil coefficients
    double *gR = nullptr, *gZ = nullptr;          // g: [kGeo][nRg], [kGeo][nZg] reconstruction factors
    // workspace
    double *Pg = nullptr, *FR = nullptr, *FZ = nullptr, *Qh = nullptr, *Pn = nullptr;
    double *SR = nullptr, *SZ = nullptr, *U = nullptr;   // g: limited slopes [4][n_s][ng], D-scaled u [n_s][ng]
};

namespace cdc {
namespace {

constexpr int NG = 2;
constexpr int kT = 256;

// Per-cell factors of the limited linear reconstruction along one direction
// (ghosted index k, centres x, edges e): inverse forward centre spacing,
// the grid factors c_F, c_B of the generalised van Leer limiter, c_F + c_B -
// 2, and the offsets of the upper and lower edge from the centre.
enum { G_IF = 0, G_CF, G_CB, G_CS, G_HI, G_LO, kGeo };

struct TView {
    int ns, nR, nZ, nRg, nZg;
    const double *Rc, *tc, *Re, *te, *sn, *cs, *V, *AR, *AZ;
    const double *gR, *gZ, *iV, *irg, *iSc;
    const double *rho_g, *nu, *Sc;     // active per cell; Sc per species
    int bc[4];
    double floor;
};

TView view(const cudisc_dust_ctx *c)
{
    TView v;
    v.ns = c->ns; v.nR = c->nR; v.nZ = c->nZ; v.nRg = c->nRg; v.nZg = c->nZg;
    v.Rc = c->Rc; v.tc = c->tc; v.Re = c->Re; v.te = c->te; v.sn = c->sn; v.cs = c->cs;
    v.V = c->V; v.AR = c->AR; v.AZ = c->AZ;
    v.gR = c->gR; v.gZ = c->gZ; v.iV = c->iV; v.irg = c->irg; v.iSc = c->iSc;
    v.rho_g = c->p.rho_g; v.nu = c->p.nu; v.Sc = c->p.Sc;
    for (int k = 0; k < 4; k++) v.bc[k] = c->p.bc[k];
    v.floor = c->p.floor;
    return v;
}

// gas of a ghosted cell: the nearest active cell's
__device__ __forceinline__ int active_cell(const TView &t, int gi, int gj)
{
    const int i = min(max(gi - NG, 0), t.nR - 1), j = min(max(gj - NG, 0), t.nZ - 1);
    return i * t.nZ + j;
}

// Ghosted primitives (rho, v_R, l, v_Z) from the active conserved field: a
// polar-side ghost of a ZERO boundary, else a radial-side ghost of one, is
// the floor density at rest; every other cell copies the nearest active cell
// (outflow and closed alike).  With diffusion, also u = rho / (rho_g Sc) per
// ghosted cell: the dust-to-gas ratio over the species' Schmidt number,
// whose differences the diffusion flux takes.
__global__ void ghost_prim_kernel(TView t, const double *__restrict__ Q, double *__restrict__ Pg,
                                  double *__restrict__ U)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    const int ng = t.nRg * t.nZg;
    if (g >= ng) return;
    const int gi = g / t.nZg, gj = g - gi * t.nZg;
    const bool zlo = gj < NG, zhi = gj >= NG + t.nZ, rlo = gi < NG, rhi = gi >= NG + t.nR;
    const bool rest = (zlo && t.bc[2] == CUDISC_BC_ZERO) || (zhi && t.bc[3] == CUDISC_BC_ZERO) ||
                      (rlo && t.bc[0] == CUDISC_BC_ZERO) || (rhi && t.bc[1] == CUDISC_BC_ZERO);
    const size_t nc = (size_t)t.nR * t.nZ, pl = (size_t)t.ns * nc, pg = (size_t)t.ns * ng;
    double rho, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    if (rest) {
        rho = t.floor;
    } else {
        const size_t e = (size_t)s * nc + active_cell(t, gi, gj);
        rho = Q[e];
        if (rho >= 1e-300) {            // 1 / rho finite: one division for the three velocities
            const double r = 1.0 / rho;
            v1 = Q[pl + e] * r;
            v2 = Q[2 * pl + e] * r;
            v3 = Q[3 * pl + e] * r;
        } else if (rho > 0.0) {
            v1 = Q[pl + e] / rho;
            v2 = Q[2 * pl + e] / rho;
            v3 = Q[3 * pl + e] / rho;
        }
    }
    const size_t o = (size_t)s * ng + g;
    if (t.nu) U[o] = rho * t.irg[active_cell(t, gi, gj)] * t.iSc[s];
    Pg[o] = rho;
    Pg[pg + o] = v1;
    Pg[2 * pg + o] = v2;
    Pg[3 * pg + o] = v3;
}

// Primitives of the source update, (rho, v_R, v_phi, v_Z) with v_phi = l / R.
__global__ void prim_kernel(int ns, int nc, const double *__restrict__ Q, const double *__restrict__ iRcell,
                            double *__restrict__ P)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (c >= nc) return;
    const size_t pl = (size_t)ns * nc, e = (size_t)s * nc + c;
    const double rho = Q[e];
    double v1 = 0.0, v2 = 0.0, v3 = 0.0;
    if (rho >= 1e-300) {
        const double r = 1.0 / rho;
        v1 = Q[pl + e] * r;
        v2 = Q[2 * pl + e] * r * iRcell[c];
        v3 = Q[3 * pl + e] * r;
    } else if (rho > 0.0) {
        v1 = Q[pl + e] / rho;
        v2 = Q[2 * pl + e] / rho * iRcell[c];
        v3 = Q[3 * pl + e] / rho;
    }
    P[e] = rho;
    P[pl + e] = v1;
    P[2 * pl + e] = v2;
    P[3 * pl + e] = v3;
}

// Generalised van Leer slope of a cell (forward and backward slopes per unit
// length between centres, grid factors c_F, c_B, cs = c_F + c_B - 2; zero at
// an extremum).
__device__ __forceinline__ double vl_slope(double sF, double sB, double cF, double cB, double cs)
{
    if (!(sF * sB > 0.0)) return 0.0;
    const double den = sB * sB + cs * sF * sB + sF * sF;
    return den != 0.0 ? sF * sB * (cF * sB + cB * sF) / den : 0.0;
}

// Limited slopes of the four primitives per ghosted cell and species, along
// R (rows NG - 1 .. NG + n_R of the active columns) and along theta (columns
// NG - 1 .. NG + n_Z of the active rows), for the
// second-order face states: each cell's slopes are computed once here rather
// than once for each of its faces in the flux kernels.
__global__ void slope_kernel(TView t, const double *__restrict__ Pg, double *__restrict__ SR,
                             double *__restrict__ SZ)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    const int ng = t.nRg * t.nZg;
    if (g >= ng) return;
    const int gi = g / t.nZg, gj = g - gi * t.nZg;
    const size_t pg = (size_t)t.ns * ng, o = (size_t)s * ng + g;
    // R slopes of the cells beside a radial face (active columns), theta
    // slopes of the cells beside a polar face (active rows)
    const bool acol = gj >= NG && gj < NG + t.nZ, arow = gi >= NG && gi < NG + t.nR;
    const bool rok = acol && gi >= NG - 1 && gi <= NG + t.nR, zok = arow && gj >= NG - 1 && gj <= NG + t.nZ;
    if (!rok && !zok) return;
    const double *gr = t.gR, *gz = t.gZ;
    const int nRg = t.nRg, nZg = t.nZg;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const double *P = Pg + q * pg + o;
        const double c = P[0];
        if (rok) {
            const double sF = (P[nZg] - c) * gr[G_IF * nRg + gi], sB = (c - P[-nZg]) * gr[G_IF * nRg + gi - 1];
            SR[q * pg + o] = vl_slope(sF, sB, gr[G_CF * nRg + gi], gr[G_CB * nRg + gi], gr[G_CS * nRg + gi]);
        }
        if (zok) {
            const double sF = (P[1] - c) * gz[G_IF * nZg + gj], sB = (c - P[-1]) * gz[G_IF * nZg + gj - 1];
            SZ[q * pg + o] = vl_slope(sF, sB, gz[G_CF * nZg + gj], gz[G_CB * nZg + gj], gz[G_CS * nZg + gj]);
        }
    }
}

// Upwind flux of the pressureless Riemann problem for face states (rho, v_R,
// l, v_Z) with normal velocities uL, uR.  The upwind side is the sign of the
// Roe-averaged velocity (sqrt(rho_L) uL + sqrt(rho_R) uR) / (sqrt(rho_L) +
// sqrt(rho_R)); only its sign is used, and that sign is fixed without the
// square roots: it is the common sign of the two terms where they agree,
// and where uL > 0 > uR the sign of rho_L uL^2 - rho_R uR^2 (both sides of
// the comparison squared).  A zero average (no mass on either side, or equal
// and opposite terms) takes the mean of the two one-sided fluxes.
__device__ __forceinline__ void riemann(const double (&L)[4], const double (&R)[4], double uL, double uR,
                                        double (&F)[4])
{
    const double rl = fmax(L[0], 0.0), rr = fmax(R[0], 0.0);
    const double tl = rl > 0.0 ? uL : 0.0, tr = rr > 0.0 ? uR : 0.0;   // signs of the two terms
    int sg;
    if (tl >= 0.0 && tr >= 0.0) sg = (tl > 0.0 || tr > 0.0) ? 1 : 0;
    else if (tl <= 0.0 && tr <= 0.0) sg = -1;
    else if (tl > 0.0) {
        const double pl = rl * uL * uL, pr = rr * uR * uR;
        sg = pl > pr ? 1 : pl < pr ? -1 : 0;
    } else sg = 0;                                 // uL < 0 < uR: the vacuum case below
    const double fl[4] = {L[0] * uL, L[0] * L[1] * uL, L[0] * L[2] * uL, L[0] * L[3] * uL};
    const double fr[4] = {R[0] * uR, R[0] * R[1] * uR, R[0] * R[2] * uR, R[0] * R[3] * uR};
    const bool vac = uL < 0.0 && uR > 0.0;
#pragma unroll
    for (int f = 0; f < 4; f++)
        F[f] = vac ? 0.0 : sg > 0 ? fl[f] : sg < 0 ? fr[f] : 0.5 * (fl[f] + fr[f]);
}

// Fluxes (per unit area) through the radial faces: thread (s, a, jj), face
// at ghosted edge i + 1 = NG + a between cells (i, j) and (i + 1, j), j =
// NG + jj.  Order 1: donor cell; order 2: the cells' limited linear states
// at the face (slopes from slope_kernel).
template <int Order>
__global__ void flux_R_kernel(TView t, const double *__restrict__ Pg, const double *__restrict__ SR,
                              const double *__restrict__ U, const double *__restrict__ cR,
                              double *__restrict__ FR)
{
    const int nf = (t.nR + 1) * t.nZ;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (f >= nf) return;
    const int a = f / t.nZ, jj = f - a * t.nZ;
    const int i = NG - 1 + a, j = NG + jj;
    const size_t ng = (size_t)t.nRg * t.nZg, pg = (size_t)t.ns * ng;
    const size_t ok = (size_t)s * ng + (size_t)i * t.nZg + j, ol = ok + t.nZg;   // cells (i, j), (i + 1, j)
    double L[4], R[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        L[q] = Pg[q * pg + ok];
        R[q] = Pg[q * pg + ol];
        if (Order == 2) {
            L[q] += SR[q * pg + ok] * t.gR[G_HI * t.nRg + i];
            R[q] += SR[q * pg + ol] * t.gR[G_LO * t.nRg + i + 1];
        }
    }
    double F[4];
    riemann(L, R, L[1], R[1], F);
    if (t.nu) {
        // partners: (i, j - 1) of the low-R cell, (i + 1, j + 1) of the high-R cell
        const double d = cR[f] * U[ok] + cR[nf + f] * U[ol] + cR[2 * nf + f] * U[ok - 1] +
                         cR[3 * nf + f] * U[ol + 1];
        const double *W = d > 0.0 ? L : R;
        F[0] += d;
        F[1] += d * W[1];
        F[2] += d * W[2];
        F[3] += d * W[3];
    }
    const bool shut = (a == 0 && t.bc[0] == CUDISC_BC_CLOSED) || (a == t.nR && t.bc[1] == CUDISC_BC_CLOSED);
    const size_t fs = (size_t)t.ns * nf, o = (size_t)s * nf + f;
#pragma unroll
    for (int q = 0; q < 4; q++) FR[q * fs + o] = shut ? 0.0 : F[q];
}

// Fluxes through the polar faces: thread (s, ii, b), face at ghosted theta
// edge j + 1 = NG + b between cells (i, j) and (i, j + 1), i = NG + ii; the
// flux is along the face normal (-sin theta^e, cos theta^e).
template <int Order>
__global__ void flux_Z_kernel(TView t, const double *__restrict__ Pg, const double *__restrict__ SZ,
                              const double *__restrict__ U, const double *__restrict__ cZ,
                              double *__restrict__ FZ)
{
    const int nf = t.nR * (t.nZ + 1);
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (f >= nf) return;
    const int ii = f / (t.nZ + 1), b = f - ii * (t.nZ + 1);
    const int i = NG + ii, j = NG - 1 + b;
    const size_t ng = (size_t)t.nRg * t.nZg, pg = (size_t)t.ns * ng;
    const size_t oa = (size_t)s * ng + (size_t)i * t.nZg + j, ol = oa + 1;       // cells (i, j), (i, j + 1)
    double L[4], R[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        L[q] = Pg[q * pg + oa];
        R[q] = Pg[q * pg + ol];
        if (Order == 2) {
            L[q] += SZ[q * pg + oa] * t.gZ[G_HI * t.nZg + j];
            R[q] += SZ[q * pg + ol] * t.gZ[G_LO * t.nZg + j + 1];
        }
    }
    const double sn = t.sn[j + 1], cs = t.cs[j + 1];
    double F[4];
    riemann(L, R, -sn * L[1] + cs * L[3], -sn * R[1] + cs * R[3], F);
    if (t.nu) {
        // partners: (i - 1, j) of the lower cell, (i + 1, j + 1) of the upper cell
        const double d = cZ[f] * U[oa] + cZ[nf + f] * U[ol] + cZ[2 * nf + f] * U[oa - t.nZg] +
                         cZ[3 * nf + f] * U[ol + t.nZg];
        const double *W = d > 0.0 ? L : R;
        F[0] += d;
        F[1] += d * W[1];
        F[2] += d * W[2];
        F[3] += d * W[3];
    }
    const bool shut = (b == 0 && t.bc[2] == CUDISC_BC_CLOSED) || (b == t.nZ && t.bc[3] == CUDISC_BC_CLOSED);
    const size_t fs = (size_t)t.ns * nf, o = (size_t)s * nf + f;
#pragma unroll
    for (int q = 0; q < 4; q++) FZ[q * fs + o] = shut ? 0.0 : F[q];
}

// Q_out = Q_base - k dt (FA) / V (Eqs. advdisc, fluxarea, halftimestepupdate).
__global__ void update_kernel(TView t, const double *__restrict__ Qb, const double *__restrict__ FR,
                              const double *__restrict__ FZ, double kdt, double *__restrict__ Qo)
{
    const int nc = t.nR * t.nZ;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (c >= nc) return;
    const int i = c / t.nZ, j = c - i * t.nZ;
    const int nfr = (t.nR + 1) * t.nZ, nfz = t.nR * (t.nZ + 1);
    const size_t pl = (size_t)t.ns * nc, fsr = (size_t)t.ns * nfr, fsz = (size_t)t.ns * nfz;
    const int r0 = i * t.nZ + j, r1 = (i + 1) * t.nZ + j;          // inner, outer radial faces
    const int z0 = i * (t.nZ + 1) + j, z1 = z0 + 1;               // lower, upper polar faces
    const double ar0 = t.AR[r0], ar1 = t.AR[r1], az0 = t.AZ[z0], az1 = t.AZ[z1];
    const double k = kdt * t.iV[c];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const double *fr = FR + q * fsr + (size_t)s * nfr, *fz = FZ + q * fsz + (size_t)s * nfz;
        const double FA = fr[r1] * ar1 - fr[r0] * ar0 + fz[z1] * az1 - fz[z0] * az0;
        const size_t e = q * pl + (size_t)s * nc + c;
        Qo[e] = Qb[e] - k * FA;
    }
}

// ---- the diffusion stencil (Sec. 3.2, Appendix A) --------------------------
struct V2 { double x, y; };
__device__ __forceinline__ V2 centre(const TView &t, int gi, int gj) { return {t.Rc[gi], t.Rc[gi] * t.tc[gj]}; }

// Interpolation point on a face line (point p0, unit normal n) between cells
// of centres x1, x2 and diffusion constants D1, D2: the projections of the
// centres weighted by w = (D / d) / sum; returns the point and w1, w2.
__device__ void interp(V2 x1, V2 x2, double D1, double D2, V2 p0, V2 n, V2 &y, double &w1, double &w2)
{
    const double s1 = (x1.x - p0.x) * n.x + (x1.y - p0.y) * n.y;
    const double s2 = (x2.x - p0.x) * n.x + (x2.y - p0.y) * n.y;
    const double a1 = D1 / fabs(s1), a2 = D2 / fabs(s2);
    w1 = a1 / (a1 + a2);
    w2 = a2 / (a1 + a2);
    y.x = w1 * (x1.x - s1 * n.x) + w2 * (x2.x - s2 * n.x);
    y.y = w1 * (x1.y - s1 * n.y) + w2 * (x2.y - s2 * n.y);
}

// c1 v1 + c2 v2 = n
__device__ __forceinline__ void solve2(V2 v1, V2 v2, V2 n, double &c1, double &c2)
{
    const double det = v1.x * v2.y - v1.y * v2.x;
    c1 = (n.x * v2.y - n.y * v2.x) / det;
    c2 = (v1.x * n.y - v1.y * n.x) / det;
}

__device__ __forceinline__ double Dcell(const TView &t, int gi, int gj)
{
    const int c = active_cell(t, gi, gj);
    return t.rho_g[c] * t.nu[c];
}

// net flux coefficients of one face from the one-sided fluxes of its two
// cells (k, its partner m across face tau; l, its partner p across face nu):
//   F_k = -D_k [w_l c_kl (u_l - u_k) + w_m c_km (u_m - u_k)],
//   F_l = -D_l [w_k c_lk (u_k - u_l) + w_p c_lp (u_p - u_l)],
//   net = w_k F_k - w_l F_l  ->  coefficients of u_k, u_l, u_m, u_p
__device__ void net_coeffs(double Dk, double Dl, double wk, double wl, double wm, double wp, double ckl,
                           double ckm, double clk, double clp, double (&o)[4])
{
    const double fk_l = -Dk * wl * ckl, fk_m = -Dk * wm * ckm;
    const double fl_k = -Dl * wk * clk, fl_p = -Dl * wp * clp;
    o[0] = wk * -(fk_l + fk_m) - wl * fl_k;
    o[1] = wk * fk_l - wl * -(fl_k + fl_p);
    o[2] = wk * fk_m;
    o[3] = -wl * fl_p;
}

// Reciprocals of the gas density per cell and of the Schmidt number per
// species, for the diffusion variable u of ghost_prim_kernel.
__global__ void gas_recip_kernel(int nc, int ns, const double *__restrict__ rho_g, const double *__restrict__ Sc,
                                 double *__restrict__ irg, double *__restrict__ iSc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nc) irg[k] = 1.0 / rho_g[k];
    if (k < ns) iSc[k] = 1.0 / Sc[k];
}

__global__ void stencil_kernel(TView t, double *__restrict__ cR, double *__restrict__ cZ)
{
    const int nfr = (t.nR + 1) * t.nZ, nfz = t.nR * (t.nZ + 1);
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < nfr) {
        // radial face at edge i + 1 between k = (i, j), l = (i + 1, j); partners
        // m = (i, j - 1) across k's lower polar face, p = (i + 1, j + 1) across
        // l's upper one
        const int a = f / t.nZ, jj = f - a * t.nZ;
        const int i = NG - 1 + a, j = NG + jj;
        const V2 xk = centre(t, i, j), xl = centre(t, i + 1, j), xm = centre(t, i, j - 1), xp = centre(t, i + 1, j + 1);
        const double Dk = Dcell(t, i, j), Dl = Dcell(t, i + 1, j), Dm = Dcell(t, i, j - 1), Dp = Dcell(t, i + 1, j + 1);
        V2 ys, yt, yn;
        double wk, wl, wkt, wm, wln, wp;
        interp(xk, xl, Dk, Dl, {t.Re[i + 1], 0.0}, {1.0, 0.0}, ys, wk, wl);
        interp(xk, xm, Dk, Dm, {0.0, 0.0}, {-t.sn[j], t.cs[j]}, yt, wkt, wm);
        interp(xl, xp, Dl, Dp, {0.0, 0.0}, {-t.sn[j + 1], t.cs[j + 1]}, yn, wln, wp);
        double ckl, ckm, clk, clp, o[4];
        solve2({ys.x - xk.x, ys.y - xk.y}, {yt.x - xk.x, yt.y - xk.y}, {1.0, 0.0}, ckl, ckm);
        solve2({ys.x - xl.x, ys.y - xl.y}, {yn.x - xl.x, yn.y - xl.y}, {-1.0, 0.0}, clk, clp);
        net_coeffs(Dk, Dl, wk, wl, wm, wp, ckl, ckm, clk, clp, o);
#pragma unroll
        for (int q = 0; q < 4; q++) cR[(size_t)q * nfr + f] = o[q];
    } else if (f < nfr + nfz) {
        // polar face at theta edge j + 1 between a = (i, j), l = (i, j + 1);
        // partners m = (i - 1, j) across a's inner radial face, b = (i + 1, j + 1)
        // across l's outer one
        const int g = f - nfr;
        const int ii = g / (t.nZ + 1), bb = g - ii * (t.nZ + 1);
        const int i = NG + ii, j = NG - 1 + bb;
        const V2 xa = centre(t, i, j), xl = centre(t, i, j + 1), xm = centre(t, i - 1, j), xb = centre(t, i + 1, j + 1);
        const double Da = Dcell(t, i, j), Dl = Dcell(t, i, j + 1), Dm = Dcell(t, i - 1, j), Db = Dcell(t, i + 1, j + 1);
        const V2 n = {-t.sn[j + 1], t.cs[j + 1]};
        V2 yl, yb, ye;
        double wa, wl, wab, wm, wle, wb;
        interp(xa, xl, Da, Dl, {0.0, 0.0}, n, yl, wa, wl);
        interp(xa, xm, Da, Dm, {t.Re[i], 0.0}, {1.0, 0.0}, yb, wab, wm);
        interp(xl, xb, Dl, Db, {t.Re[i + 1], 0.0}, {1.0, 0.0}, ye, wle, wb);
        double cal, cam, cla, clb, o[4];
        solve2({yl.x - xa.x, yl.y - xa.y}, {yb.x - xa.x, yb.y - xa.y}, n, cal, cam);
        solve2({yl.x - xl.x, yl.y - xl.y}, {ye.x - xl.x, ye.y - xl.y}, {-n.x, -n.y}, cla, clb);
        net_coeffs(Da, Dl, wa, wl, wm, wb, cal, cam, cla, clb, o);
#pragma unroll
        for (int q = 0; q < 4; q++) cZ[(size_t)q * nfz + g] = o[q];
    }
}

// ---- host geometry ----------------------------------------------------------
std::vector<double> extend_edges(const double *e, int n)
{
    // n + 1 edges -> n + 5: ghost cells mirror the widths of the boundary cells
    std::vector<double> w(n);
    for (int k = 0; k < n; k++) w[k] = e[k + 1] - e[k];
    std::vector<double> o(n + 5);
    const double w1 = n > 1 ? w[1] : w[0], wn2 = n > 1 ? w[n - 2] : w[0];
    o[1] = e[0] - w[0];
    o[0] = o[1] - w1;
    for (int k = 0; k <= n; k++) o[k + 2] = e[k];
    o[n + 3] = e[n] + w[n - 1];
    o[n + 4] = o[n + 3] + wn2;
    return o;
}

std::vector<double> extend_centres(const double *c, const double *e, int n)
{
    // ghost centres mirror the centres of the boundary cells across the boundary
    std::vector<double> o(n + 4);
    o[1] = 2.0 * e[0] - c[0];
    o[0] = n > 1 ? 2.0 * e[0] - c[1] : o[1] - (e[1] - e[0]);
    for (int k = 0; k < n; k++) o[k + 2] = c[k];
    o[n + 2] = 2.0 * e[n] - c[n - 1];
    o[n + 3] = n > 1 ? 2.0 * e[n] - c[n - 2] : o[n + 2] + (e[n] - e[n - 1]);
    return o;
}

// Reconstruction factors along one ghosted direction of n cells (centres x,
// edges e): G_IF at k = 1 / (x[k + 1] - x[k]) (k < n - 1), and at cells
// 1 .. n - 2 the limiter's c_F = (x[k + 1] - x[k]) / (e[k + 1] - x[k]),
// c_B = (x[k] - x[k - 1]) / (x[k] - e[k]), c_F + c_B - 2, and the edge
// offsets e[k + 1] - x[k], e[k] - x[k].
std::vector<double> recon_factors(const std::vector<double> &x, const std::vector<double> &e)
{
    const int n = (int)x.size();
    std::vector<double> g((size_t)kGeo * n, 0.0);
    for (int k = 0; k + 1 < n; k++) g[G_IF * n + k] = 1.0 / (x[k + 1] - x[k]);
    for (int k = 1; k + 1 < n; k++) {
        const double cF = (x[k + 1] - x[k]) / (e[k + 1] - x[k]), cB = (x[k] - x[k - 1]) / (x[k] - e[k]);
        g[G_CF * n + k] = cF;
        g[G_CB * n + k] = cB;
        g[G_CS * n + k] = cF + cB - 2.0;
    }
    for (int k = 0; k < n; k++) {
        g[G_HI * n + k] = e[k + 1] - x[k];
        g[G_LO * n + k] = e[k] - x[k];
    }
    return g;
}

template <class T> cudaError_t up(T **d, const std::vector<T> &h, cudaStream_t s)
{
    cudaError_t e = cudaMalloc(d, h.size() * sizeof(T));
    if (e == cudaSuccess) e = cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    return e;
}

dim3 grid2(size_t n, int y) { return dim3((unsigned)((n + kT - 1) / kT), (unsigned)y); }

} // namespace
} // namespace cdc

using namespace cdc;

static void free_dust(cudisc_dust_ctx *c)
{
    if (!c) return;
    double *ptrs[] = {c->Rc, c->tc, c->Re, c->te, c->sn, c->cs, c->V, c->AR, c->AZ, c->Rcell, c->Zcell,
                      c->iV, c->iRcell, c->irg, c->iSc, c->cR, c->cZ, c->gR, c->gZ, c->Pg, c->FR, c->FZ, c->Qh, c->Pn, c->SR, c->SZ, c->U};
    for (double *q : ptrs)
        if (q) cudaFree(q);
    delete c;
}

static cudisc_status dust_fail(cudisc_dust_ctx *c, cudisc_status st, const std::string &msg)
{
    if (c) c->err = msg;
    cdc::set_thread_error(msg);
    return st;
}

#define DUST_TRY(ctx, expr)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return dust_fail(ctx, e_ == cudaErrorMemoryAllocation ? CUDISC_ENOMEM : CUDISC_ECUDA, \
                             std::string(#expr ": ") + cudaGetErrorString(e_));                \
    } while (0)

extern "C" {

cudisc_status cudisc_dust_init(const cudisc_dust_params *p, cudisc_dust_ctx **out)
{
    cdc::set_thread_error("");
    if (!out) return dust_fail(nullptr, CUDISC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p) return dust_fail(nullptr, CUDISC_EINVAL, "params is NULL");
    if (p->n_species < 1 || p->n_species > 65535 || p->n_R < 1 || p->n_Z < 1 ||
        (long long)p->n_R * p->n_Z > (1ll << 30) ||
        (long long)p->n_species * (p->n_R + 4) * (p->n_Z + 4) > (1ll << 31))
        return dust_fail(nullptr, CUDISC_EINVAL, "n_species (<= 65535), n_R and n_Z must be >= 1 (and not huge)");
    if (!p->R_e || !p->th_e) return dust_fail(nullptr, CUDISC_EINVAL, "R_e and th_e must be host arrays");
    if (!p->rho_g) return dust_fail(nullptr, CUDISC_EINVAL, "rho_g must be a device array");
    if (p->nu && !p->Sc) return dust_fail(nullptr, CUDISC_EINVAL, "Sc must be given with nu");
    if (p->c_s && (!p->v_g || !p->a)) return dust_fail(nullptr, CUDISC_EINVAL, "sources need c_s, v_g and a");
    if (p->c_s && (!(p->rho_m > 0.0) || !(p->GM >= 0.0)))
        return dust_fail(nullptr, CUDISC_EINVAL, "sources need rho_m > 0 and GM >= 0");
    if (p->geometry != CUDISC_GEOM_CYLINDRICAL && p->geometry != CUDISC_GEOM_CARTESIAN)
        return dust_fail(nullptr, CUDISC_EINVAL, "geometry must be CUDISC_GEOM_CYLINDRICAL or _CARTESIAN");
    for (int k = 0; k < 4; k++)
        if (p->bc[k] < CUDISC_BC_OUTFLOW || p->bc[k] > CUDISC_BC_ZERO)
            return dust_fail(nullptr, CUDISC_EINVAL, "bc entries must be OUTFLOW, CLOSED or ZERO");
    const int nR = p->n_R, nZ = p->n_Z;
    for (int k = 0; k < nR; k++)
        if (!(p->R_e[k + 1] > p->R_e[k]) || !(p->R_e[k] > 0.0))
            return dust_fail(nullptr, CUDISC_EINVAL, "R_e must be positive and strictly increasing");
    for (int k = 0; k < nZ; k++)
        if (!(p->th_e[k + 1] > p->th_e[k]) || !(fabs(p->th_e[k]) < 1.5) || !(fabs(p->th_e[k + 1]) < 1.5))
            return dust_fail(nullptr, CUDISC_EINVAL, "th_e must be strictly increasing within (-1.5, 1.5) rad");
    std::vector<double> Rc(nR), thc(nZ);
    for (int k = 0; k < nR; k++) Rc[k] = p->R_c ? p->R_c[k] : 0.5 * (p->R_e[k] + p->R_e[k + 1]);
    for (int k = 0; k < nZ; k++) thc[k] = p->th_c ? p->th_c[k] : 0.5 * (p->th_e[k] + p->th_e[k + 1]);
    for (int k = 0; k < nR; k++)
        if (!(Rc[k] > p->R_e[k] && Rc[k] < p->R_e[k + 1])) return dust_fail(nullptr, CUDISC_EINVAL, "R_c outside its cell");
    for (int k = 0; k < nZ; k++)
        if (!(thc[k] > p->th_e[k] && thc[k] < p->th_e[k + 1]))
            return dust_fail(nullptr, CUDISC_EINVAL, "th_c outside its cell");
    std::vector<double> Re = extend_edges(p->R_e, nR), the = extend_edges(p->th_e, nZ);
    std::vector<double> Rcg = extend_centres(Rc.data(), p->R_e, nR), thcg = extend_centres(thc.data(), p->th_e, nZ);
    if (!(Re[0] > 0.0)) return dust_fail(nullptr, CUDISC_EINVAL, "the inner ghost cells would reach R <= 0");
    if (!(fabs(the[0]) < 1.55) || !(fabs(the[nZ + 4]) < 1.55))
        return dust_fail(nullptr, CUDISC_EINVAL, "the polar ghost cells would reach |theta| >= 1.55");
    const int nRg = nR + 2 * NG, nZg = nZ + 2 * NG;
    std::vector<double> te(nZg + 1), sn(nZg + 1), cs(nZg + 1), tc(nZg);
    for (int k = 0; k <= nZg; k++) { te[k] = tan(the[k]); sn[k] = sin(the[k]); cs[k] = cos(the[k]); }
    for (int k = 0; k < nZg; k++) tc[k] = tan(thcg[k]);
    const bool cyl = p->geometry == CUDISC_GEOM_CYLINDRICAL;
    std::vector<double> V((size_t)nR * nZ), AR((size_t)(nR + 1) * nZ), AZ((size_t)nR * (nZ + 1));
    std::vector<double> Rcell((size_t)nR * nZ), Zcell((size_t)nR * nZ);
    for (int i = 0; i < nR; i++) {
        const double r0 = Re[i + NG], r1 = Re[i + NG + 1];
        const double dR = r1 - r0, dR2 = r1 * r1 - r0 * r0, dR3 = r1 * r1 * r1 - r0 * r0 * r0;
        for (int j = 0; j < nZ; j++) {
            const double dt = te[j + NG + 1] - te[j + NG];
            V[(size_t)i * nZ + j] = cyl ? dR3 / 3.0 * dt : dR2 / 2.0 * dt;
            Rcell[(size_t)i * nZ + j] = Rcg[i + NG];
            Zcell[(size_t)i * nZ + j] = Rcg[i + NG] * tc[j + NG];
        }
        for (int j = 0; j <= nZ; j++)
            AZ[(size_t)i * (nZ + 1) + j] = (cyl ? dR2 / 2.0 : dR) / cs[j + NG];
    }
    for (int a = 0; a <= nR; a++) {
        const double r = Re[a + NG];
        for (int j = 0; j < nZ; j++)
            AR[(size_t)a * nZ + j] = (cyl ? r * r : r) * (te[j + NG + 1] - te[j + NG]);
    }
    cudisc_dust_ctx *c = new cudisc_dust_ctx();
    c->p = *p;
    c->p.R_e = c->p.th_e = c->p.R_c = c->p.th_c = nullptr;   // host arrays are not kept
    c->stream = (cudaStream_t)p->stream;
    c->ns = p->n_species; c->nR = nR; c->nZ = nZ; c->nRg = nRg; c->nZg = nZg;
    cudaError_t e = cudaSuccess;
    auto U = [&](double **d, const std::vector<double> &h) { if (e == cudaSuccess) e = up(d, h, c->stream); };
    U(&c->Rc, Rcg); U(&c->tc, tc); U(&c->Re, Re); U(&c->te, te); U(&c->sn, sn); U(&c->cs, cs);
    U(&c->V, V); U(&c->AR, AR); U(&c->AZ, AZ); U(&c->Rcell, Rcell); U(&c->Zcell, Zcell);
    U(&c->gR, recon_factors(Rcg, Re)); U(&c->gZ, recon_factors(tc, te));
    {
        std::vector<double> iV(V.size()), iRc(Rcell.size());
        for (size_t k = 0; k < V.size(); k++) { iV[k] = 1.0 / V[k]; iRc[k] = 1.0 / Rcell[k]; }
        U(&c->iV, iV); U(&c->iRcell, iRc);
    }
    const size_t nc = (size_t)nR * nZ, ns = c->ns;
    const size_t nfr = (size_t)(nR + 1) * nZ, nfz = (size_t)nR * (nZ + 1);
    auto A = [&](double **d, size_t n) { if (e == cudaSuccess) e = cudaMalloc(d, n * sizeof(double)); };
    A(&c->cR, 4 * nfr); A(&c->cZ, 4 * nfz);
    A(&c->Pg, 4 * ns * (size_t)nRg * nZg); A(&c->FR, 4 * ns * nfr); A(&c->FZ, 4 * ns * nfz);
    A(&c->Qh, 4 * ns * nc); A(&c->Pn, 4 * ns * nc);
    A(&c->SR, 4 * ns * (size_t)nRg * nZg); A(&c->SZ, 4 * ns * (size_t)nRg * nZg);
    if (p->nu) { A(&c->U, ns * (size_t)nRg * nZg); A(&c->irg, nc); A(&c->iSc, ns); }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        const cudisc_status st = e == cudaErrorMemoryAllocation ? CUDISC_ENOMEM : CUDISC_ECUDA;
        const std::string m = std::string("cudisc_dust_init: ") + cudaGetErrorString(e);
        free_dust(c);
        return dust_fail(nullptr, st, m);
    }
    const cudisc_status st = cudisc_dust_update_gas(c);
    if (st != CUDISC_OK) {
        const std::string m = c->err;
        free_dust(c);
        return dust_fail(nullptr, st, m);
    }
    *out = c;
    return CUDISC_OK;
}

cudisc_status cudisc_dust_update_gas(cudisc_dust_ctx *c)
{
    if (!c) return dust_fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!c->p.nu) return CUDISC_OK;
    const TView t = view(c);
    const size_t nc = (size_t)c->nR * c->nZ, nr = nc > (size_t)c->ns ? nc : (size_t)c->ns;
    gas_recip_kernel<<<(unsigned)((nr + kT - 1) / kT), kT, 0, c->stream>>>((int)nc, c->ns, c->p.rho_g, c->p.Sc,
                                                                         c->irg, c->iSc);
    const size_t nf = (size_t)(c->nR + 1) * c->nZ + (size_t)c->nR * (c->nZ + 1);
    stencil_kernel<<<(unsigned)((nf + kT - 1) / kT), kT, 0, c->stream>>>(t, c->cR, c->cZ);
    DUST_TRY(c, cudaGetLastError());
    return CUDISC_OK;
}

cudisc_status cudisc_dust_step(cudisc_dust_ctx *c, double *Q, double dt)
{
    if (!c) return dust_fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!Q) return dust_fail(c, CUDISC_EINVAL, "Q is NULL");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return dust_fail(c, CUDISC_EINVAL, "dt must be >= 0 and finite");
    const TView t = view(c);
    const int ns = c->ns;
    const size_t nc = (size_t)c->nR * c->nZ, ng = (size_t)c->nRg * c->nZg;
    const size_t nfr = (size_t)(c->nR + 1) * c->nZ, nfz = (size_t)c->nR * (c->nZ + 1);
    const bool src = c->p.c_s != nullptr;
    cudaStream_t s = c->stream;
    // stage 1: donor-cell fluxes at n, half step, half-step sources
    ghost_prim_kernel<<<grid2(ng, ns), kT, 0, s>>>(t, Q, c->Pg, c->U);
    if (src) prim_kernel<<<grid2(nc, ns), kT, 0, s>>>(ns, (int)nc, Q, c->iRcell, c->Pn);
    flux_R_kernel<1><<<grid2(nfr, ns), kT, 0, s>>>(t, c->Pg, c->SR, c->U, c->cR, c->FR);
    flux_Z_kernel<1><<<grid2(nfz, ns), kT, 0, s>>>(t, c->Pg, c->SZ, c->U, c->cZ, c->FZ);
    update_kernel<<<grid2(nc, ns), kT, 0, s>>>(t, Q, c->FR, c->FZ, 0.5 * dt, c->Qh);
    DUST_TRY(c, cudaGetLastError());
    if (src)
        DUST_TRY(c, launch_dust_source(ns, (int)nc, c->Qh, c->Pn, 0.5 * dt, c->Rcell, c->Zcell, c->p.rho_g, c->p.c_s,
                                       c->p.v_g, c->p.a, c->p.rho_m, c->p.GM, s));
    // stage 2: limited linear fluxes at n + 1/2, full step, full-step sources
    ghost_prim_kernel<<<grid2(ng, ns), kT, 0, s>>>(t, c->Qh, c->Pg, c->U);
    if (src) prim_kernel<<<grid2(nc, ns), kT, 0, s>>>(ns, (int)nc, c->Qh, c->iRcell, c->Pn);
    slope_kernel<<<grid2(ng, ns), kT, 0, s>>>(t, c->Pg, c->SR, c->SZ);
    flux_R_kernel<2><<<grid2(nfr, ns), kT, 0, s>>>(t, c->Pg, c->SR, c->U, c->cR, c->FR);
    flux_Z_kernel<2><<<grid2(nfz, ns), kT, 0, s>>>(t, c->Pg, c->SZ, c->U, c->cZ, c->FZ);
    update_kernel<<<grid2(nc, ns), kT, 0, s>>>(t, Q, c->FR, c->FZ, dt, Q);
    DUST_TRY(c, cudaGetLastError());
    if (src)
        DUST_TRY(c, launch_dust_source(ns, (int)nc, Q, c->Pn, dt, c->Rcell, c->Zcell, c->p.rho_g, c->p.c_s,
                                       c->p.v_g, c->p.a, c->p.rho_m, c->p.GM, s));
    return CUDISC_OK;
}

cudisc_status cudisc_dust_geometry(const cudisc_dust_ctx *c, double *V, double *AR, double *AZ)
{
    if (!c) return dust_fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    const size_t nc = (size_t)c->nR * c->nZ;
    const size_t nfr = (size_t)(c->nR + 1) * c->nZ, nfz = (size_t)c->nR * (c->nZ + 1);
    cudisc_dust_ctx *m = const_cast<cudisc_dust_ctx *>(c);
    if (V) DUST_TRY(m, cudaMemcpyAsync(V, c->V, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (AR) DUST_TRY(m, cudaMemcpyAsync(AR, c->AR, nfr * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (AZ) DUST_TRY(m, cudaMemcpyAsync(AZ, c->AZ, nfz * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    DUST_TRY(m, cudaStreamSynchronize(c->stream));
    return CUDISC_OK;
}

void cudisc_dust_destroy(cudisc_dust_ctx *c) { free_dust(c); }

} // extern "C"
