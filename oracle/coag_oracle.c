/*
 * coag_oracle.c -- plain, slow FP64 CPU oracle of the per-cell
 * Smoluchowski coagulation-fragmentation update of Sec. 5 of
 * Robinson, Booth & Owen, "Introducing cuDisc" (arXiv 2402.18471).
 *
 * TEST INFRASTRUCTURE.  Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; the only common input is
 * the seeded synthetic disc built in Python.
 *
 * Every function follows the paper's definitions in its order and notation,
 * with plain loops and no blocking or reordering:
 *   Eq. (smol)            rho_dot_k = sum_i sum_{j<=i} gain_ijk - sum_i loss_ik
 *   loss                  loss_ik = m_k n_i n_k K_ik (p_coag + p_frag = 1)
 *   Eq. (kernel)          K_ij = sigma_ij dv_ij, sigma_ij = pi (a_i + a_j)^2
 *   dv^2 = v_BM^2 + v_turb^2 + dv_lam^2
 *   Eq. (vbrown)          v_BM = sqrt(8 k_B T (m_i + m_j) / (pi m_i m_j))
 *   v_turb = sqrt(alpha) c_s V_rel, Eq. (OCVrel) with Ormel & Cuzzi (2007)
 *                         class I / class II closed forms
 *   Eq. (ngain)           gain with C_ijk, R_ijk, F_ijk; K -> K/2 at i = j
 *   Eq. (p_frag)          p_frag = (1.5 (v_f/dv)^2 + 1) exp(-1.5 (v_f/dv)^2)
 *   Eqs. (Cijk), (Rijk)   two-bin split with eps(m) = (m_u - m)/(m_u - m_l)
 *   Eqs. (fragdist), (Nijk) fragment power law and N_k(m_max)
 *   Eq. (fragrem)         remnant mass; fragment mass = total - remnant
 *   Sec. 5 last paragraph Bogacki-Shampine 3(2), rtol 1e-2, atol 1e-10 sum rho
 *   Eq. (t_stop)          Epstein stopping time, v_th = sqrt(8/pi) c_s
 *   Sec. 3.3              nu = alpha c_s H; Re = nu_t / nu_mol (Sec. 7.2)
 *   adjoint               the paper has none: the discrete adjoint of the
 *                         replayed BS3 map (step sizes frozen), written out
 *                         stage by stage from the forward formulas above
 *
 * Readings where the paper is silent or ambiguous (each is listed with its
 * reason in the design notes):
 *   - l(m) = max{k : m_k <= m}, u = l + 1; an exact grid hit puts all mass in k.
 *   - products above the top bin go wholly to bin N-1; remnants below bin 0
 *     wholly to bin 0 (mass conserving).
 *   - split_mode 0: C, R are literal MASS fractions eps, 1 - eps (the paper's
 *     wording); split_mode 1: number fractions (mass and number conserving).
 *   - the largest-fragment bin l uses m_x = min(chi m_im, m_tar); the mass
 *     distributed as fragments is m_i + m_j - m_rem.
 *   - loss uses the full K (no 1/2 at i = j); with the 1/2 on the gain side
 *     this conserves mass exactly.
 *   - St* = min(max(1.6 St_1, Re^-1/2), 1) (OC07 intermediate-regime ratio
 *     in place of the unprinted quadratic fit); the class II term integrates
 *     the per-particle response 1 - St^2/(St + t)^2 of BOTH particles, which
 *     reproduces OC07's tiny, intermediate (their Eq. 28) and heavy limits.
 *   - nu_mol = v_th lambda_mfp / 2, lambda_mfp = mu m_H / (rho_g sigma_H2).
 *   - laminar dv from input dust velocities, or terminal drift/settling
 *     velocities v_R = -2 eta v_K St/(1+St^2), v_phi = -eta v_K/(1+St^2),
 *     v_Z = -Z Omega St/(1+St), with v_K = Omega R.
 *   - vertically integrated kernel (Sec. 5.1, the 1D comparison with a
 *     surface-density code): states are surface densities, the cell is a
 *     radius (Z unused, Omega = Omega_mid, rho_gas = mid-plane density),
 *     grain scale heights h = H sqrt(alpha / (alpha + St)), settling
 *     velocities v_Z = -h Omega St/(1+St) (each grain at its own scale
 *     height), and K -> K / sqrt(2 pi (h_i^2 + h_j^2)).
 *   - integrator: per-cell step, max-norm error, safety 0.9, factor clamp
 *     [0.2, 5], reject on y' < -atol, first step 0.1 min (|y|+atol)/|f|.
 *
 * Parity status of each exported function is stated next to it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n_cells, n_bins;
    const double *m;        /* [N]   bin-centre masses */
    const double *me;       /* [N+1] bin edges */
    const double *rho_gas;  /* [n_cells] */
    const double *T;
    const double *alpha;
    const double *R;
    const double *Z;
    const double *eta;      /* drift parameter, may be NULL (no drift) */
    const double *v_dust;   /* [3][n_cells][N] or NULL */
    double v_frag, eta_frag, chi_im, rho_m, mu, Mstar;
    double k_B, m_H, G, sigma_H2;
    double kernel_const;
    int kernel_mode;        /* 0 physical, 1 constant, 2 additive */
    int frag_mode;          /* 0 physical p_frag, 1 never, 2 always */
    int split_mode;         /* 0 mass fraction, 1 number fraction */
    int n_threads;          /* <= 0: library default */
    double rtol, atol_rel;
    long max_substeps;
    int vertical;           /* 1: vertically integrated kernel (Sec. 5.1) */
    /* Sensitivity runs only (not part of the method): K_ij (1 + kernel_perturb
     * u) and, in replays, every stage input y_k (1 + stage_noise u), u uniform
     * in [-1/2, 1/2), drawn per (perturb_seed, cell, pair) and per
     * (perturb_seed, cell, step, stage, bin). */
    double kernel_perturb;
    unsigned long long perturb_seed;
    double stage_noise;
} oracle_params;

enum { ST_OK = 0, ST_MAXSTEPS = 4, ST_NONFINITE = 5, ST_DTMIN = 7 };

/* ------------------------------------------------------------------------ */
/* Two-bin split of a product mass (Eqs. Cijk, Rijk) with the readings above */
/* ------------------------------------------------------------------------ */
static void split_mass(const oracle_params *P, double mass, int *kl, int *ku,
                       double *fl, double *fu)
{
    const int N = P->n_bins;
    const double *m = P->m;
    if (mass >= m[N - 1]) { *kl = *ku = N - 1; *fl = 1.0; *fu = 0.0; return; }
    if (mass <= m[0])     { *kl = *ku = 0;     *fl = 1.0; *fu = 0.0; return; }
    int l = 0;
    for (int k = 0; k < N; k++) if (m[k] <= mass) l = k;   /* largest m_l <= m */
    int u = l + 1;
    double eps = (m[u] - mass) / (m[u] - m[l]);
    *kl = l; *ku = u;
    if (P->split_mode == 1) {           /* number fractions -> mass fractions */
        *fl = eps * m[l] / mass;
        *fu = (1.0 - eps) * m[u] / mass;
    } else {                            /* literal mass fractions */
        *fl = eps;
        *fu = 1.0 - eps;
    }
}

/* N_k(m_max), Eq. (Nijk), for k <= l with m_max = me[l+1]. */
static double frag_fraction(const oracle_params *P, int k, double mmax)
{
    const double *me = P->me;
    double s = 2.0 - P->eta_frag;
    if (fabs(s) < 1e-12)
        return log(me[k + 1] / me[k]) / log(mmax / me[0]);
    return (pow(me[k + 1], s) - pow(me[k], s)) / (pow(mmax, s) - pow(me[0], s));
}

/* Remnant and fragment masses of pair (i, j), Eq. (fragrem). */
static void remnant(const oracle_params *P, int i, int j, double *mrem,
                    double *mfrag_total, int *l_frag)
{
    const double *m = P->m, *me = P->me;
    const int N = P->n_bins;
    double mtar = m[i] > m[j] ? m[i] : m[j];
    double mim = m[i] > m[j] ? m[j] : m[i];
    double chi_mim = P->chi_im * mim;
    double mr = (chi_mim < mtar) ? (mtar - chi_mim) : 0.0;
    double mx = chi_mim < mtar ? chi_mim : mtar;     /* largest fragment */
    int l = N - 1;
    for (int q = N - 1; q >= 0; q--) if (me[q + 1] > mx) l = q; /* smallest */
    *mrem = mr;
    *mfrag_total = m[i] + m[j] - mr;
    *l_frag = l;
}

/* ------------------------------------------------------------------------ */
/* Relative velocities and the collision kernel                             */
/* ------------------------------------------------------------------------ */

/* Ormel & Cuzzi (2007) V_rel^2 in units of V_g^2 = alpha c_s^2.
 * St1 >= St2 are the larger and smaller Stokes numbers, delta = Re^-1/2. */
double oracle_vrel2(double Sa, double Sb, double Re)
{
    double S1 = Sa > Sb ? Sa : Sb;
    double S2 = Sa > Sb ? Sb : Sa;
    double d = 1.0 / sqrt(Re);
    double Ss = 1.6 * S1;
    if (Ss < d) Ss = d;
    if (Ss > 1.0) Ss = 1.0;
    /* class I (slow eddies, t* .. t_L) */
    double dVI = 0.0;
    if (S1 + S2 > 0.0)
        dVI = (S1 - S2) / (S1 + S2) *
              (S1 * S1 / (Ss + S1) - S1 * S1 / (1.0 + S1)
               - S2 * S2 / (Ss + S2) + S2 * S2 / (1.0 + S2));
    /* class II (fast eddies, t_eta .. t*), both particles' responses */
    double dVII = 2.0 * (Ss - d)
                + S1 * S1 / (S1 + Ss) - S1 * S1 / (S1 + d)
                + S2 * S2 / (S2 + Ss) - S2 * S2 / (S2 + d);
    double v = dVI + dVII;
    return v > 0.0 ? v : 0.0;
}

double oracle_pfrag(double dv, double vf)
{
    if (!(dv > 0.0)) return 0.0;
    double x = 1.5 * (vf / dv) * (vf / dv);
    return (x + 1.0) * exp(-x);
}

/* Per-cell, per-bin quantities: sizes, Stokes numbers, dust velocities. */
typedef struct {
    double cs, Re, Vg2, T;
    double *a, *St, *vR, *vphi, *vZ, *h;   /* h: grain scale heights (vertical mode) */
    int cell;
} cellphys;

/* SplitMix64 finaliser (Steele, Lea & Flood 2014) of a counter: a uniform
 * number in [-1/2, 1/2) for the sensitivity runs. */
static double counter_uniform(unsigned long long seed, unsigned long long a, unsigned long long b,
                              unsigned long long c)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (1ull + a);
    z ^= b * 0xD1B54A32D192ED03ull;
    z += c * 0x8CB92BA72F3D8DD7ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

static void cell_physics(const oracle_params *P, int c, cellphys *cp)
{
    const int N = P->n_bins;
    double T = P->T[c], rg = P->rho_gas[c], R = P->R[c], Z = P->vertical ? 0.0 : P->Z[c];
    double cs = sqrt(P->k_B * T / (P->mu * P->m_H));
    double vth = sqrt(8.0 / M_PI) * cs;
    double r2 = R * R + Z * Z;
    double Omega = sqrt(P->G * P->Mstar / (r2 * sqrt(r2)));
    double Omega_mid = sqrt(P->G * P->Mstar / (R * R * R));
    double H = cs / Omega_mid;
    double nu_t = P->alpha[c] * cs * H;
    double lmfp = P->mu * P->m_H / (rg * P->sigma_H2);
    double nu_mol = 0.5 * vth * lmfp;
    cp->cs = cs;
    cp->cell = c;
    cp->Re = nu_t / nu_mol;
    cp->Vg2 = P->alpha[c] * cs * cs;
    cp->T = T;
    double eta = P->eta ? P->eta[c] : 0.0;
    double vK = Omega * R;
    for (int k = 0; k < N; k++) {
        double a = cbrt(3.0 * P->m[k] / (4.0 * M_PI * P->rho_m));
        double ts = P->rho_m * a / (rg * vth);
        double St = ts * Omega;
        cp->a[k] = a;
        cp->St[k] = St;
        /* dust scale height of a Gaussian layer stirred by turbulence */
        cp->h[k] = P->vertical ? H * sqrt(P->alpha[c] / (P->alpha[c] + St)) : 0.0;
        if (P->v_dust) {
            size_t nc = (size_t)P->n_cells * N;
            cp->vR[k] = P->v_dust[(size_t)c * N + k];
            cp->vphi[k] = P->v_dust[nc + (size_t)c * N + k];
            cp->vZ[k] = P->v_dust[2 * nc + (size_t)c * N + k];
        } else {
            cp->vR[k] = -2.0 * eta * vK * St / (1.0 + St * St);
            cp->vphi[k] = -eta * vK / (1.0 + St * St);
            /* settling at the height Z, or at the grain's own scale height */
            double zk = P->vertical ? cp->h[k] : Z;
            cp->vZ[k] = -zk * Omega * St / (1.0 + St);
        }
    }
}

/* Kernel and fragmentation probability of pair (i, j) in a cell. */
static void pair_kernel(const oracle_params *P, const cellphys *cp, int i, int j,
                        double *K, double *pf, double *dv_out)
{
    const double *m = P->m;
    double vbm2 = 8.0 * P->k_B * cp->T * (m[i] + m[j]) / (M_PI * m[i] * m[j]);
    double vt2 = cp->Vg2 * oracle_vrel2(cp->St[i], cp->St[j], cp->Re);
    double dR = cp->vR[i] - cp->vR[j];
    double dP = cp->vphi[i] - cp->vphi[j];
    double dZ = cp->vZ[i] - cp->vZ[j];
    double vl2 = dR * dR + dP * dP + dZ * dZ;
    double dv = sqrt(vbm2 + vt2 + vl2);
    double s = cp->a[i] + cp->a[j];
    double k;
    if (P->kernel_mode == 1) k = P->kernel_const;
    else if (P->kernel_mode == 2) k = P->kernel_const * (m[i] + m[j]);
    else k = M_PI * s * s * dv;
    /* vertically integrated: the rate of two Gaussian layers per unit area */
    if (P->vertical) k /= sqrt(2.0 * M_PI * (cp->h[i] * cp->h[i] + cp->h[j] * cp->h[j]));
    if (P->kernel_perturb != 0.0) {   /* sensitivity runs only, symmetric in i, j */
        const int a = i > j ? i : j, b = i > j ? j : i;
        k *= 1.0 + P->kernel_perturb * counter_uniform(P->perturb_seed, (unsigned long long)cp->cell,
                                                       (unsigned long long)a, (unsigned long long)b);
    }
    double p;
    if (P->frag_mode == 1) p = 0.0;
    else if (P->frag_mode == 2) p = 1.0;
    else p = oracle_pfrag(dv, P->v_frag);
    *K = k; *pf = p;
    if (dv_out) *dv_out = dv;
}

/* ------------------------------------------------------------------------ */
/* Per-cell data: K and p_frag matrices (constant during a step call).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ckl, cku, rkl, rku, l;        /* coag split, remnant split, frag bin */
    double cfl, cfu, rfl, rfu, mrem, mfr;
} pairmap;

typedef struct {
    const oracle_params *P;
    int c;
    double *K, *pf;      /* [N*N] full symmetric */
    double *flag;        /* [N] fragment mass per largest-fragment bin */
    pairmap *map;        /* [N*N], entries j <= i: Eqs. (Cijk), (Rijk), (fragrem) */
    double *Ntab;        /* [N*N] N_k(m^e_{l+1}), row l (Eq. Nijk) */
} cellctx;

static void *xmalloc(size_t n) { void *p = calloc(n ? n : 1, 1); return p; }

static void cell_alloc(const oracle_params *P, int c, cellctx *cx)
{
    const int N = P->n_bins;
    cellphys cp;
    double *buf = xmalloc(sizeof(double) * 6 * N);
    cp.a = buf; cp.St = buf + N; cp.vR = buf + 2 * N; cp.vphi = buf + 3 * N;
    cp.vZ = buf + 4 * N; cp.h = buf + 5 * N;
    cell_physics(P, c, &cp);
    cx->P = P; cx->c = c;
    cx->K = xmalloc(sizeof(double) * N * N);
    cx->pf = xmalloc(sizeof(double) * N * N);
    cx->flag = xmalloc(sizeof(double) * N);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            pair_kernel(P, &cp, i, j, &cx->K[i * N + j], &cx->pf[i * N + j], NULL);
    free(buf);
    /* the mapping coefficients do not change during a call: evaluate once */
    cx->map = xmalloc(sizeof(pairmap) * N * N);
    cx->Ntab = xmalloc(sizeof(double) * N * N);
    for (int i = 0; i < N; i++)
        for (int j = 0; j <= i; j++) {
            pairmap *q = &cx->map[i * N + j];
            split_mass(P, P->m[i] + P->m[j], &q->ckl, &q->cku, &q->cfl, &q->cfu);
            remnant(P, i, j, &q->mrem, &q->mfr, &q->l);
            if (q->mrem > 0.0) split_mass(P, q->mrem, &q->rkl, &q->rku, &q->rfl, &q->rfu);
            else { q->rkl = q->rku = 0; q->rfl = q->rfu = 0.0; }
        }
    for (int l = 0; l < N; l++)
        for (int k = 0; k <= l; k++) cx->Ntab[l * N + k] = frag_fraction(P, k, P->me[l + 1]);
}

static void cell_free(cellctx *cx)
{
    free(cx->K); free(cx->pf); free(cx->flag); free(cx->map); free(cx->Ntab);
}

/* Eq. (smol) for one cell, with fragments gathered per largest-fragment bin l
 * and then distributed by N_k(m^e_{l+1}) (the two-stage form of Sec. 5). */
static void rhs_cell(void *vctx, const double *rho, double *drho)
{
    cellctx *cx = vctx;
    const oracle_params *P = cx->P;
    const int N = P->n_bins;
    const double *m = P->m;
    for (int k = 0; k < N; k++) { drho[k] = 0.0; cx->flag[k] = 0.0; }
    for (int i = 0; i < N; i++) {
        double ni = rho[i] / m[i];
        for (int j = 0; j <= i; j++) {
            double nj = rho[j] / m[j];
            double K = cx->K[i * N + j];
            double pf = cx->pf[i * N + j];
            double pc = 1.0 - pf;
            double W = ni * nj * K;
            if (i == j) W *= 0.5;
            const pairmap *q = &cx->map[i * N + j];
            /* coagulation product of mass m_i + m_j */
            double mc = m[i] + m[j];
            drho[q->ckl] += W * pc * mc * q->cfl;
            drho[q->cku] += W * pc * mc * q->cfu;
            /* remnant and fragments */
            if (q->mrem > 0.0) {
                drho[q->rkl] += W * pf * q->mrem * q->rfl;
                drho[q->rku] += W * pf * q->mrem * q->rfu;
            }
            cx->flag[q->l] += W * pf * q->mfr;
            /* loss: the pair removes one grain of each colliding species */
            drho[i] -= W * m[i];
            drho[j] -= W * m[j];
        }
    }
    for (int l = 0; l < N; l++) {
        if (cx->flag[l] == 0.0) continue;
        for (int k = 0; k <= l; k++) drho[k] += cx->flag[l] * cx->Ntab[l * N + k];
    }
}

static int nthreads_of(const oracle_params *P)
{
#ifdef _OPENMP
    return P->n_threads > 0 ? P->n_threads : omp_get_max_threads();
#else
    (void)P; return 1;
#endif
}

/* ========================================================================
 * Exported functions
 * ====================================================================== */

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Per-cell diagnostics for tests: St[N], a[N], velocities, grain scale
 * heights h[N] (vertical mode; zeros otherwise) and {cs, Re, Vg2}.
 * Parity: pinned (Stokes / Epstein closed forms are re-derived in tests;
 * h by its small- and large-St limits and the vertical integral of the
 * volume rate). */
int oracle_cell_physics(const oracle_params *P, int c, double *a, double *St,
                        double *vR, double *vphi, double *vZ, double *h, double *scal3)
{
    cellphys cp; cp.a = a; cp.St = St; cp.vR = vR; cp.vphi = vphi; cp.vZ = vZ; cp.h = h;
    cell_physics(P, c, &cp);
    scal3[0] = cp.cs; scal3[1] = cp.Re; scal3[2] = cp.Vg2;
    return 0;
}

/* Full K and p_frag matrices [n_cells][N][N] and dv [n_cells][N][N].
 * Parity: pinned (Brownian by Monte Carlo, OC07 limits, p_frag as a Gamma
 * survival function, symmetry). */
int oracle_kernel(const oracle_params *P, double *K, double *pf, double *dv)
{
    const int N = P->n_bins;
    #pragma omp parallel for schedule(dynamic) num_threads(nthreads_of(P))
    for (int c = 0; c < P->n_cells; c++) {
        cellphys cp;
        double *buf = xmalloc(sizeof(double) * 6 * N);
        cp.a = buf; cp.St = buf + N; cp.vR = buf + 2 * N; cp.vphi = buf + 3 * N;
        cp.vZ = buf + 4 * N; cp.h = buf + 5 * N;
        cell_physics(P, c, &cp);
        size_t o = (size_t)c * N * N;
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++)
                pair_kernel(P, &cp, i, j, &K[o + i * N + j], &pf[o + i * N + j],
                            dv ? &dv[o + i * N + j] : NULL);
        free(buf);
    }
    return 0;
}

/* Mapping of one pair: coag split, remnant split, fragment bin and masses.
 * out_i[5] = {c_l, c_u, r_l, r_u, l}; out_d[6] = {c_fl, c_fu, r_fl, r_fu,
 * m_rem, m_frag_total}.  Parity: pinned (mass placed = mass produced). */
int oracle_pair_map(const oracle_params *P, int i, int j, int *out_i, double *out_d)
{
    int kl, ku, l; double fl, fu, mrem, mfr;
    split_mass(P, P->m[i] + P->m[j], &kl, &ku, &fl, &fu);
    out_i[0] = kl; out_i[1] = ku; out_d[0] = fl; out_d[1] = fu;
    remnant(P, i, j, &mrem, &mfr, &l);
    if (mrem > 0.0) split_mass(P, mrem, &kl, &ku, &fl, &fu);
    else { kl = ku = 0; fl = fu = 0.0; }
    out_i[2] = kl; out_i[3] = ku; out_i[4] = l;
    out_d[2] = fl; out_d[3] = fu; out_d[4] = mrem; out_d[5] = mfr;
    return 0;
}

/* N_k(m^e_{l+1}) table [N][N] (row l, column k), zero for k > l.
 * Parity: pinned (quadrature of the power law, Eq. fragdist). */
int oracle_frag_table(const oracle_params *P, double *tab)
{
    const int N = P->n_bins;
    for (int l = 0; l < N; l++)
        for (int k = 0; k < N; k++)
            tab[l * N + k] = (k <= l) ? frag_fraction(P, k, P->me[l + 1]) : 0.0;
    return 0;
}

/* rho_dot for every cell (two-stage fragment form).  Parity: pinned
 * (mass conservation, brute-force triple sum, closed-form kernels). */
int oracle_rhs(const oracle_params *P, const double *rho, double *drho)
{
    const int N = P->n_bins;
    #pragma omp parallel for schedule(dynamic) num_threads(nthreads_of(P))
    for (int c = 0; c < P->n_cells; c++) {
        cellctx cx;
        cell_alloc(P, c, &cx);
        rhs_cell(&cx, rho + (size_t)c * N, drho + (size_t)c * N);
        cell_free(&cx);
    }
    return 0;
}

/* Brute-force Eq. (smol): dense C_ijk, R_ijk, F_ijk tensors, gain summed over
 * i, j <= i, k with F_ijk = N_k(m_max,ij) applied pair by pair, and the loss
 * written as m_k n_i n_k K_ik summed over all i.  Tiny grids only. */
int oracle_rhs_bruteforce(const oracle_params *P, const double *rho, double *drho)
{
    const int N = P->n_bins;
    const double *m = P->m;
    double *C = xmalloc(sizeof(double) * N * N * N);
    double *Rt = xmalloc(sizeof(double) * N * N * N);
    double *F = xmalloc(sizeof(double) * N * N * N);
    double *mrem = xmalloc(sizeof(double) * N * N);
    double *mfr = xmalloc(sizeof(double) * N * N);
    for (int i = 0; i < N; i++)
        for (int j = 0; j <= i; j++) {
            int kl, ku, l; double fl, fu, mr, mf;
            split_mass(P, m[i] + m[j], &kl, &ku, &fl, &fu);
            C[(i * N + j) * N + kl] += fl;
            C[(i * N + j) * N + ku] += fu;
            remnant(P, i, j, &mr, &mf, &l);
            mrem[i * N + j] = mr; mfr[i * N + j] = mf;
            if (mr > 0.0) {
                split_mass(P, mr, &kl, &ku, &fl, &fu);
                Rt[(i * N + j) * N + kl] += fl;
                Rt[(i * N + j) * N + ku] += fu;
            }
            for (int k = 0; k <= l; k++)
                F[(i * N + j) * N + k] = frag_fraction(P, k, P->me[l + 1]);
        }
    for (int c = 0; c < P->n_cells; c++) {
        cellctx cx;
        cell_alloc(P, c, &cx);
        const double *r = rho + (size_t)c * N;
        double *d = drho + (size_t)c * N;
        for (int k = 0; k < N; k++) {
            double gain = 0.0, loss = 0.0;
            for (int i = 0; i < N; i++) {
                double ni = r[i] / m[i];
                for (int j = 0; j <= i; j++) {
                    double nj = r[j] / m[j];
                    double K = cx.K[i * N + j];
                    if (i == j) K *= 0.5;
                    double pf = cx.pf[i * N + j], pc = 1.0 - pf;
                    size_t t = (size_t)(i * N + j) * N + k;
                    gain += ni * nj * K * (pc * (m[i] + m[j]) * C[t]
                            + pf * (mrem[i * N + j] * Rt[t] + mfr[i * N + j] * F[t]));
                }
                loss += m[k] * ni * (r[k] / m[k]) * cx.K[i * N + k];
            }
            d[k] = gain - loss;
        }
        cell_free(&cx);
    }
    free(C); free(Rt); free(F); free(mrem); free(mfr);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Bogacki-Shampine 3(2) with per-cell step-size control                    */
/* ------------------------------------------------------------------------ */
typedef void (*rhs_fn)(void *ctx, const double *y, double *f);

static const double BS_A21 = 0.5, BS_A32 = 0.75;
static const double BS_B1 = 2.0 / 9.0, BS_B2 = 1.0 / 3.0, BS_B3 = 4.0 / 9.0;
static const double BS_E1 = -5.0 / 72.0, BS_E2 = 1.0 / 12.0, BS_E3 = 1.0 / 9.0,
                    BS_E4 = -1.0 / 8.0;

typedef struct {
    long n_acc, n_rej;
    int status;
    double h_last;
} bs3_stats;

static int bs3_integrate(rhs_fn f, void *ctx, int n, double *y, double t_span,
                         double h, double rtol, double atol, long max_steps,
                         double *log, long log_cap, long *n_log, bs3_stats *st)
{
    double *k1 = xmalloc(sizeof(double) * n), *k2 = xmalloc(sizeof(double) * n);
    double *k3 = xmalloc(sizeof(double) * n), *k4 = xmalloc(sizeof(double) * n);
    double *Y = xmalloc(sizeof(double) * n), *y1 = xmalloc(sizeof(double) * n);
    long nl = 0;
    st->n_acc = st->n_rej = 0; st->status = ST_OK;
    double t = 0.0;
    f(ctx, y, k1);
    if (!(h > 0.0)) {
        double hmin = INFINITY;
        for (int k = 0; k < n; k++)
            if (k1[k] != 0.0) {
                double q = (fabs(y[k]) + atol) / fabs(k1[k]);
                if (q < hmin) hmin = q;
            }
        h = isfinite(hmin) ? 0.1 * hmin : t_span;
        if (h > t_span) h = t_span;
    }
    while (t < t_span) {
        if (st->n_acc + st->n_rej >= max_steps) { st->status = ST_MAXSTEPS; break; }
        int last = (h >= t_span - t);
        double hs = last ? (t_span - t) : h;
        for (int k = 0; k < n; k++) Y[k] = y[k] + hs * BS_A21 * k1[k];
        f(ctx, Y, k2);
        for (int k = 0; k < n; k++) Y[k] = y[k] + hs * BS_A32 * k2[k];
        f(ctx, Y, k3);
        for (int k = 0; k < n; k++)
            y1[k] = y[k] + hs * (BS_B1 * k1[k] + BS_B2 * k2[k] + BS_B3 * k3[k]);
        f(ctx, y1, k4);
        double E = 0.0, ymin = INFINITY;
        int finite = 1;
        for (int k = 0; k < n; k++) {
            double e = hs * (BS_E1 * k1[k] + BS_E2 * k2[k] + BS_E3 * k3[k] + BS_E4 * k4[k]);
            double sc = atol + rtol * fmax(fabs(y[k]), fabs(y1[k]));
            /* an empty cell has atol = 0 and y = 0: no error, not 0/0 */
            double r = (e == 0.0) ? 0.0 : fabs(e) / sc;
            if (!isfinite(r) || !isfinite(y1[k])) finite = 0;
            if (r > E) E = r;
            if (y1[k] < ymin) ymin = y1[k];
        }
        if (finite && E <= 1.0 && ymin >= -atol) {
            t = last ? t_span : t + hs;
            memcpy(y, y1, sizeof(double) * n);
            memcpy(k1, k4, sizeof(double) * n);
            st->n_acc++;
            if (log && nl < log_cap) log[nl] = hs;
            nl++;
            double fac = (E > 0.0) ? 0.9 * pow(E, -1.0 / 3.0) : 5.0;
            if (fac > 5.0) fac = 5.0;
            if (fac < 0.2) fac = 0.2;
            if (!(last && hs < h)) h = hs * fac;
        } else {
            st->n_rej++;
            double fac;
            if (!finite) fac = 0.2;
            else if (E > 1.0) { fac = 0.9 * pow(E, -1.0 / 3.0); if (fac < 0.2) fac = 0.2; }
            else fac = 0.5;
            h = hs * fac;
            /* a step that keeps shrinking after rejections has failed */
            if (h < 1e-14 * t_span) { st->status = finite ? ST_DTMIN : ST_NONFINITE; break; }
        }
    }
    st->h_last = h;
    if (n_log) *n_log = nl;
    free(k1); free(k2); free(k3); free(k4); free(Y); free(y1);
    return st->status;
}

static void bs3_fixed(rhs_fn f, void *ctx, int n, double *y, const double *hs, long nh)
{
    double *k1 = xmalloc(sizeof(double) * n), *k2 = xmalloc(sizeof(double) * n);
    double *k3 = xmalloc(sizeof(double) * n), *Y = xmalloc(sizeof(double) * n);
    for (long s = 0; s < nh; s++) {
        double h = hs[s];
        f(ctx, y, k1);
        for (int k = 0; k < n; k++) Y[k] = y[k] + h * BS_A21 * k1[k];
        f(ctx, Y, k2);
        for (int k = 0; k < n; k++) Y[k] = y[k] + h * BS_A32 * k2[k];
        f(ctx, Y, k3);
        for (int k = 0; k < n; k++)
            y[k] = y[k] + h * (BS_B1 * k1[k] + BS_B2 * k2[k] + BS_B3 * k3[k]);
    }
    free(k1); free(k2); free(k3); free(Y);
}

/* Adaptive coagulation step of every cell c over its span: spans[c] when
 * spans is given (a cell with spans[c] <= 0 is not touched: no steps,
 * status 0, dt[c] kept), else t_span for all cells.
 * dt[c]: in = first step (<= 0: automatic), out = last proposed step.
 * Optional per-cell logs of accepted steps: dt_log[c*log_cap + s]. */
static int step_cells(const oracle_params *P, double *rho, double t_span, const double *spans,
                      double *dt, long *n_acc, long *n_rej, int *status, double *dt_log,
                      long log_cap, long *n_log)
{
    const int N = P->n_bins;
    int worst = 0;
    #pragma omp parallel for schedule(dynamic) num_threads(nthreads_of(P)) reduction(max:worst)
    for (int c = 0; c < P->n_cells; c++) {
        const double span = spans ? spans[c] : t_span;
        if (!(span > 0.0)) {
            if (n_acc) n_acc[c] = 0;
            if (n_rej) n_rej[c] = 0;
            if (status) status[c] = 0;
            if (n_log) n_log[c] = 0;
            continue;
        }
        cellctx cx;
        cell_alloc(P, c, &cx);
        double *y = rho + (size_t)c * N;
        double s = 0.0;
        for (int k = 0; k < N; k++) s += y[k];
        double atol = P->atol_rel * s;
        bs3_stats st;
        long nl = 0;
        bs3_integrate(rhs_cell, &cx, N, y, span, dt ? dt[c] : 0.0, P->rtol, atol,
                      P->max_substeps, dt_log ? dt_log + (size_t)c * log_cap : NULL,
                      log_cap, &nl, &st);
        if (dt) dt[c] = st.h_last;
        if (n_acc) n_acc[c] = st.n_acc;
        if (n_rej) n_rej[c] = st.n_rej;
        if (status) status[c] = st.status;
        if (n_log) n_log[c] = nl;
        if (st.status > worst) worst = st.status;
        cell_free(&cx);
    }
    return worst;
}

/* Every cell over t_span.  Parity: pinned (closed-form constant/additive
 * kernels, BS3 order tests). */
int oracle_step(const oracle_params *P, double *rho, double t_span, double *dt,
                long *n_acc, long *n_rej, int *status, double *dt_log,
                long log_cap, long *n_log)
{
    return step_cells(P, rho, t_span, NULL, dt, n_acc, n_rej, status, dt_log, log_cap, n_log);
}

/* Cell c over spans[c] (cells with spans[c] <= 0 untouched): the update of
 * the cells that a sub-cycled global step (Sec. 6) brings up to date.
 * Parity: pinned as oracle_step (a single-cell span equals a whole-grid
 * step of that span; skipped cells are bitwise unchanged). */
int oracle_step_spans(const oracle_params *P, double *rho, const double *spans, double *dt,
                      long *n_acc, long *n_rej, int *status, double *dt_log,
                      long log_cap, long *n_log)
{
    return step_cells(P, rho, 0.0, spans, dt, n_acc, n_rej, status, dt_log, log_cap, n_log);
}

/* Replay: apply a given sequence of accepted BS3 steps to every cell
 * (hs[c*stride + s], s < n_h[c]).  Parity: pinned as oracle_step. */
/* The replay of bs3_fixed with every stage input perturbed by a relative
 * stage_noise u (sensitivity runs only): the same three stages, each right-
 * hand side evaluated at Y_k (1 + stage_noise u). */
static void bs3_fixed_noisy(cellctx *cx, int n, double *y, const double *hs, long nh)
{
    const oracle_params *P = cx->P;
    double *k1 = xmalloc(sizeof(double) * n), *k2 = xmalloc(sizeof(double) * n);
    double *k3 = xmalloc(sizeof(double) * n), *Y = xmalloc(sizeof(double) * n);
    for (long s = 0; s < nh; s++) {
        double h = hs[s];
        for (int st = 0; st < 3; st++) {
            for (int k = 0; k < n; k++) {
                double v = st == 0 ? y[k] : st == 1 ? y[k] + h * BS_A21 * k1[k] : y[k] + h * BS_A32 * k2[k];
                Y[k] = v * (1.0 + P->stage_noise * counter_uniform(P->perturb_seed, (unsigned long long)cx->c,
                                                                    (unsigned long long)(3 * s + st),
                                                                    (unsigned long long)k + 0x100000000ull));
            }
            rhs_cell(cx, Y, st == 0 ? k1 : st == 1 ? k2 : k3);
        }
        for (int k = 0; k < n; k++)
            y[k] = y[k] + h * (BS_B1 * k1[k] + BS_B2 * k2[k] + BS_B3 * k3[k]);
    }
    free(k1); free(k2); free(k3); free(Y);
}

int oracle_step_replay(const oracle_params *P, double *rho, const double *hs,
                       const long *n_h, long stride)
{
    const int N = P->n_bins;
    #pragma omp parallel for schedule(dynamic) num_threads(nthreads_of(P))
    for (int c = 0; c < P->n_cells; c++) {
        cellctx cx;
        cell_alloc(P, c, &cx);
        if (P->stage_noise != 0.0)
            bs3_fixed_noisy(&cx, N, rho + (size_t)c * N, hs + (size_t)c * stride, n_h[c]);
        else
            bs3_fixed(rhs_cell, &cx, N, rho + (size_t)c * N, hs + (size_t)c * stride, n_h[c]);
        cell_free(&cx);
    }
    return 0;
}

/* Scalar test problem y' = lam y through the same stepper (order checks).
 * mode 0: adaptive over t_span from h0; mode 1: n_fixed steps of h0.
 * out[0] = y(t_span), out[1] = accepted, out[2] = rejected. */
typedef struct { double lam; } lin_ctx;
static void lin_rhs(void *c, const double *y, double *f) { f[0] = ((lin_ctx *)c)->lam * y[0]; }

int oracle_bs3_scalar(double lam, double y0, double t_span, double h0, double rtol,
                      double atol, int mode, long n_fixed, double *out)
{
    lin_ctx cx = { lam };
    double y = y0;
    if (mode == 1) {
        double *hs = xmalloc(sizeof(double) * (n_fixed ? n_fixed : 1));
        for (long s = 0; s < n_fixed; s++) hs[s] = h0;
        bs3_fixed(lin_rhs, &cx, 1, &y, hs, n_fixed);
        free(hs);
        out[0] = y; out[1] = (double)n_fixed; out[2] = 0.0;
        return 0;
    }
    bs3_stats st;
    bs3_integrate(lin_rhs, &cx, 1, &y, t_span, h0, rtol, atol, 100000000L, NULL, 0, NULL, &st);
    out[0] = y; out[1] = (double)st.n_acc; out[2] = (double)st.n_rej;
    return st.status;
}

/* ======================================================================== */
/* Discrete adjoint of the replayed step sequence                           */
/* ======================================================================== */

/* Derivatives of K_ij and p_frag,ij with respect to alpha (turbulent term,
 * including Re = nu_t / nu_mol proportional to alpha in delta = Re^-1/2 and
 * in the St* clamp) and of p_frag with respect to v_frag. */
static void pair_kernel_deriv(const oracle_params *P, const cellphys *cp, int c, int i, int j,
                              double *dK_da, double *dpf_da, double *dpf_dvf)
{
    const double *m = P->m;
    double alpha = P->alpha[c];
    double K, pf, dv;
    pair_kernel(P, cp, i, j, &K, &pf, &dv);
    double S1 = cp->St[i] > cp->St[j] ? cp->St[i] : cp->St[j];
    double S2 = cp->St[i] > cp->St[j] ? cp->St[j] : cp->St[i];
    double d = 1.0 / sqrt(cp->Re);
    double a16 = 1.6 * S1;
    double Ss = a16 < d ? d : a16;
    int clamp_d = (a16 < d) && (d < 1.0);
    if (Ss > 1.0) Ss = 1.0;
    double V = oracle_vrel2(cp->St[i], cp->St[j], cp->Re);
    double dVI_dSs = 0.0;
    if (S1 + S2 > 0.0)
        dVI_dSs = (S1 - S2) / (S1 + S2) *
                  (-S1 * S1 / ((Ss + S1) * (Ss + S1)) + S2 * S2 / ((Ss + S2) * (Ss + S2)));
    double dVII_dSs = 2.0 - S1 * S1 / ((S1 + Ss) * (S1 + Ss)) - S2 * S2 / ((S2 + Ss) * (S2 + Ss));
    double dVII_dd = -2.0 + S1 * S1 / ((S1 + d) * (S1 + d)) + S2 * S2 / ((S2 + d) * (S2 + d));
    double dV_dd = (dVI_dSs + dVII_dSs) * (clamp_d ? 1.0 : 0.0) + dVII_dd;
    if (!(V > 0.0)) dV_dd = 0.0;
    double cs2 = cp->cs * cp->cs;
    double dd_da = -0.5 * d / alpha;                 /* delta ~ alpha^-1/2 */
    double dvt2_da = cs2 * V + alpha * cs2 * dV_dd * dd_da;
    /* vertically integrated kernel: h = H sqrt(alpha / (alpha + St)) gives
     * dh/dalpha = h g with g = St / (2 alpha (alpha + St)); the settling
     * velocities -h Omega St/(1+St) scale with h, and the factor
     * f = (2 pi (h_i^2 + h_j^2))^-1/2 has d ln f / dalpha =
     * -(h_i^2 g_i + h_j^2 g_j) / (h_i^2 + h_j^2) */
    double gi = 0.0, gj = 0.0;
    if (P->vertical) {
        gi = cp->St[i] / (2.0 * alpha * (alpha + cp->St[i]));
        gj = cp->St[j] / (2.0 * alpha * (alpha + cp->St[j]));
        if (!P->v_dust) {
            double dZ = cp->vZ[i] - cp->vZ[j];
            dvt2_da += 2.0 * dZ * (cp->vZ[i] * gi - cp->vZ[j] * gj);
        }
    }
    double ddv_da = dv > 0.0 ? dvt2_da / (2.0 * dv) : 0.0;
    double s = cp->a[i] + cp->a[j];
    *dK_da = (P->kernel_mode == 0) ? M_PI * s * s * ddv_da : 0.0;
    if (P->vertical) {
        double hi2 = cp->h[i] * cp->h[i], hj2 = cp->h[j] * cp->h[j];
        double f = 1.0 / sqrt(2.0 * M_PI * (hi2 + hj2));
        double dlnf = -(hi2 * gi + hj2 * gj) / (hi2 + hj2);
        *dK_da = f * *dK_da + K * dlnf;              /* K includes f */
    }
    double dpf_ddv = 0.0, dpfdvf = 0.0;
    if (P->frag_mode == 0 && dv > 0.0) {
        double x = 1.5 * (P->v_frag / dv) * (P->v_frag / dv);
        dpf_ddv = 2.0 * x * x * exp(-x) / dv;
        dpfdvf = -2.0 * x * x * exp(-x) / P->v_frag;
    }
    *dpf_da = dpf_ddv * ddv_da;
    *dpf_dvf = dpfdvf;
    (void)m; (void)K; (void)pf;
}

/* ybar += J(rho)^T v and the per-pair cotangents of K (Kbar) and p_frag
 * (pfbar), for the right-hand side of rhs_cell written pair by pair. */
static void rhs_vjp_cell(cellctx *cx, const double *rho, const double *v, double *ybar,
                         double *Kbar, double *pfbar, double *Fv)
{
    const oracle_params *P = cx->P;
    const int N = P->n_bins;
    const double *m = P->m;
    for (int l = 0; l < N; l++) {
        double t = 0.0;
        for (int k = 0; k <= l; k++) t += v[k] * cx->Ntab[l * N + k];
        Fv[l] = t;
    }
    for (int i = 0; i < N; i++) {
        double ni = rho[i] / m[i];
        for (int j = 0; j <= i; j++) {
            double nj = rho[j] / m[j];
            double h = (i == j) ? 0.5 : 1.0;
            double K = cx->K[i * N + j];
            double pf = cx->pf[i * N + j];
            const pairmap *q = &cx->map[i * N + j];
            double mc = m[i] + m[j];
            double Gc = mc * (q->cfl * v[q->ckl] + q->cfu * v[q->cku]);
            double Gr = (q->mrem > 0.0) ? q->mrem * (q->rfl * v[q->rkl] + q->rfu * v[q->rku]) : 0.0;
            double Gf = q->mfr * Fv[q->l];
            double Gl = -(m[i] * v[i] + m[j] * v[j]);
            double G = (1.0 - pf) * Gc + pf * (Gr + Gf) + Gl;
            double W = ni * nj * K * h;
            ybar[i] += G * nj * K * h / m[i];
            ybar[j] += G * ni * K * h / m[j];
            Kbar[i * N + j] += G * ni * nj * h;
            pfbar[i * N + j] += W * (Gr + Gf - Gc);
        }
    }
}

/* Gradient of L = sum_{c,k} w[c][k] rho_ck(T), where rho(T) is reached from
 * rho0 by the given accepted BS3 steps (hs[c*stride + s], s < n_h[c]; the
 * step sequence is held fixed), with respect to rho0 (g_rho0 [c][k]), the
 * per-cell alpha (g_alpha [c], may be NULL) and v_frag (*g_vfrag, summed
 * over cells, may be NULL).  Parity: pinned (central finite differences of
 * oracle_step_replay, dot-product identity). */
int oracle_vjp(const oracle_params *P, const double *rho0, const double *hs, const long *n_h,
               long stride, const double *w, double *g_rho0, double *g_alpha, double *g_vfrag)
{
    const int N = P->n_bins;
    double vf_total = 0.0;
    #pragma omp parallel for schedule(dynamic) num_threads(nthreads_of(P)) reduction(+:vf_total)
    for (int c = 0; c < P->n_cells; c++) {
        cellctx cx;
        cell_alloc(P, c, &cx);
        long nh = n_h[c];
        const double *hc = hs + (size_t)c * stride;
        double *Ys = xmalloc(sizeof(double) * N * (nh + 1));
        double *k1 = xmalloc(sizeof(double) * N), *k2 = xmalloc(sizeof(double) * N);
        double *Y2 = xmalloc(sizeof(double) * N), *Y3 = xmalloc(sizeof(double) * N);
        double *lam = xmalloc(sizeof(double) * N), *yb = xmalloc(sizeof(double) * N);
        double *kb1 = xmalloc(sizeof(double) * N), *kb2 = xmalloc(sizeof(double) * N);
        double *kb3 = xmalloc(sizeof(double) * N), *Fv = xmalloc(sizeof(double) * N);
        double *Kbar = xmalloc(sizeof(double) * N * N), *pfbar = xmalloc(sizeof(double) * N * N);
        memcpy(Ys, rho0 + (size_t)c * N, sizeof(double) * N);
        for (long s = 0; s < nh; s++) {           /* forward: store every state */
            memcpy(Ys + (s + 1) * N, Ys + s * N, sizeof(double) * N);
            bs3_fixed(rhs_cell, &cx, N, Ys + (s + 1) * N, hc + s, 1);
        }
        memcpy(lam, w + (size_t)c * N, sizeof(double) * N);
        for (long s = nh - 1; s >= 0; s--) {
            const double *y = Ys + s * N;
            double h = hc[s];
            rhs_cell(&cx, y, k1);
            for (int k = 0; k < N; k++) Y2[k] = y[k] + h * BS_A21 * k1[k];
            rhs_cell(&cx, Y2, k2);
            for (int k = 0; k < N; k++) Y3[k] = y[k] + h * BS_A32 * k2[k];
            /* y' = y + h (b1 k1 + b2 k2 + b3 k3(Y3)) */
            for (int k = 0; k < N; k++) {
                yb[k] = lam[k];
                kb1[k] = h * BS_B1 * lam[k];
                kb2[k] = h * BS_B2 * lam[k];
                kb3[k] = h * BS_B3 * lam[k];
            }
            /* k3 = f(Y3), Y3 = y + h A32 k2 */
            double *Yb = xmalloc(sizeof(double) * N);
            for (int k = 0; k < N; k++) Yb[k] = 0.0;
            rhs_vjp_cell(&cx, Y3, kb3, Yb, Kbar, pfbar, Fv);
            for (int k = 0; k < N; k++) { yb[k] += Yb[k]; kb2[k] += h * BS_A32 * Yb[k]; Yb[k] = 0.0; }
            /* k2 = f(Y2), Y2 = y + h A21 k1 */
            rhs_vjp_cell(&cx, Y2, kb2, Yb, Kbar, pfbar, Fv);
            for (int k = 0; k < N; k++) { yb[k] += Yb[k]; kb1[k] += h * BS_A21 * Yb[k]; Yb[k] = 0.0; }
            /* k1 = f(y) */
            rhs_vjp_cell(&cx, y, kb1, Yb, Kbar, pfbar, Fv);
            for (int k = 0; k < N; k++) lam[k] = yb[k] + Yb[k];
            free(Yb);
        }
        memcpy(g_rho0 + (size_t)c * N, lam, sizeof(double) * N);
        /* parameters: chain the accumulated pair cotangents */
        cellphys cp;
        double *buf = xmalloc(sizeof(double) * 6 * N);
        cp.a = buf; cp.St = buf + N; cp.vR = buf + 2 * N; cp.vphi = buf + 3 * N; cp.vZ = buf + 4 * N;
        cp.h = buf + 5 * N;
        cell_physics(P, c, &cp);
        double ga = 0.0, gv = 0.0;
        for (int i = 0; i < N; i++)
            for (int j = 0; j <= i; j++) {
                double dK, dpa, dpv;
                pair_kernel_deriv(P, &cp, c, i, j, &dK, &dpa, &dpv);
                ga += Kbar[i * N + j] * dK + pfbar[i * N + j] * dpa;
                gv += pfbar[i * N + j] * dpv;
            }
        if (g_alpha) g_alpha[c] = ga;
        vf_total += gv;
        free(buf);
        free(Ys); free(k1); free(k2); free(Y2); free(Y3); free(lam); free(yb);
        free(kb1); free(kb2); free(kb3); free(Fv); free(Kbar); free(pfbar);
        cell_free(&cx);
    }
    if (g_vfrag) *g_vfrag = vf_total;
    return 0;
}
