/*
 * cudisc_coag.h -- C ABI of the B300 coagulation-fragmentation step.
 *
 * The library integrates, for every cell of an (R, Z) grid independently, the
 * Smoluchowski equation in mass-density form (Sec. 5, Eq. smol of Robinson,
 * Booth & Owen, "Introducing cuDisc", arXiv 2402.18471):
 *
 *   d rho_k / dt = sum_i sum_{j<=i} gain_ijk - sum_i m_k n_i n_k K_ik,
 *
 * with the collision kernel K_ij = pi (a_i + a_j)^2 dv_ij (Eq. kernel), the
 * relative velocity dv^2 = v_BM^2 + v_turb^2 + dv_lam^2 (Brownian, Eq. vbrown;
 * turbulent after Ormel & Cuzzi 2007, Eq. OCVrel; laminar drift/settling),
 * the fragmentation probability of Eq. (p_frag), the two-bin split of
 * coagulation products and remnants (Eqs. Cijk, Rijk, fragrem) and the
 * power-law fragment distribution (Eqs. fragdist, Nijk), gathered per
 * largest-fragment bin and then distributed.  Time integration is the
 * Bogacki-Shampine 3(2) embedded pair with per-cell adaptive steps and the
 * paper's tolerances (rtol 1e-2, atol 1e-10 x sum_k rho_k; Sec. 5, last
 * paragraph).
 *
 * Conventions
 *   - CGS units.  Cell c, bin k: dust densities are rho[c * N + k] (bins
 *     contiguous).  N = n_bins, Np = N (N + 1) / 2 pairs.
 *   - "device" arrays are CUDA global-memory pointers on the current device;
 *     "host" arrays are ordinary CPU memory.  Every array passed in stays
 *     owned by the caller; the library never frees it.  The context owns its
 *     own device buffers (kernel tables, mapping tensors, workspace).
 *   - Every call returns a cudisc_status; no call aborts or throws.  On an
 *     error cudisc_coag_last_error(ctx) returns a message (NULL ctx: the last
 *     error of the calling thread).
 *   - Work is issued on params.stream (NULL: the legacy default stream).
 *     cudisc_coag_rhs, cudisc_coag_build_kernel_async and
 *     cudisc_coag_step_async are asynchronous (and may be captured in a CUDA
 *     graph); so is cudisc_hse_rho_gas, on the stream it
 *     is given.  cudisc_coag_step, cudisc_coag_step_wait,
 *     cudisc_coag_step_spans, cudisc_coag_subcycle,
 *     cudisc_coag_subcycle_pending, cudisc_coag_build_kernel and
 *     cudisc_coag_vjp synchronise that stream before returning so they can
 *     report per-cell failures.
 */
#ifndef CUDISC_COAG_H
#define CUDISC_COAG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cudisc_coag_ctx cudisc_coag_ctx;   /* opaque, owned by the library */

typedef enum {
    CUDISC_OK = 0,
    CUDISC_EINVAL = 1,      /* bad argument: the message names it */
    CUDISC_ENOMEM = 2,      /* a device or host allocation failed */
    CUDISC_ECUDA = 3,       /* a CUDA runtime error (message has the CUDA text) */
    CUDISC_EMAXSTEPS = 4,   /* some cell hit max_substeps before t_span */
    CUDISC_ENONFINITE = 5,  /* some cell produced a non-finite state */
    CUDISC_ENOTSUP = 6,     /* size or mode outside what this build supports */
    CUDISC_EDTMIN = 7       /* some cell's step shrank below 1e-14 t_span */
} cudisc_status;

typedef enum {
    CUDISC_FP64 = 0,        /* FP64 everywhere: sparse gather on CUDA cores */
    CUDISC_MIXED_TF32 = 1   /* gain/loss contraction on tcgen05 tensor cores with
                               TF32 hi+lo split operands (4 products: hi.hi,
                               hi.lo, lo.hi, lo.lo), FP32 accumulation in TMEM
                               with compensated chunk sums, FP32 stage
                               arithmetic, FP64 state and mass budget */
} cudisc_precision;

/* Arithmetic of the adjoint's per-pair work (cudisc_coag_set_adjoint_precision). */
typedef enum {
    CUDISC_ADJOINT_FP64 = 0,          /* FP64 (the default) */
    CUDISC_ADJOINT_DOUBLE_FLOAT = 1   /* pairs of FP32 numbers (h + l, ~48
                                         significant bits, FP32 exponent range)
                                         on the FP32 pipes */
} cudisc_adjoint_precision;

typedef enum {
    CUDISC_KERNEL_PHYSICAL = 0,  /* K = pi (a_i + a_j)^2 dv (Eq. kernel) */
    CUDISC_KERNEL_CONSTANT = 1,  /* K = kernel_const (closed-form tests) */
    CUDISC_KERNEL_ADDITIVE = 2   /* K = kernel_const (m_i + m_j) */
} cudisc_kernel_mode;

typedef enum {
    CUDISC_FRAG_PHYSICAL = 0,    /* p_frag from Eq. (p_frag) */
    CUDISC_FRAG_NONE = 1,        /* p_frag = 0 */
    CUDISC_FRAG_ALL = 2          /* p_frag = 1 */
} cudisc_frag_mode;

typedef enum {
    CUDISC_SPLIT_MASS = 0,       /* C_ijk, R_ijk = eps, 1 - eps as mass fractions */
    CUDISC_SPLIT_NUMBER = 1      /* eps as the number fraction (conserves number) */
} cudisc_split_mode;

typedef struct {
    int n_cells;                 /* >= 1 */
    int n_bins;                  /* N, 2 <= N <= 160 */
    const double *mass_centres;  /* host [N], strictly increasing, g */
    const double *mass_edges;    /* host [N+1], strictly increasing,
                                    edge k < centre k < edge k+1, g */
    const double *rho_gas;       /* device [n_cells], g cm^-3 */
    const double *T;             /* device [n_cells], K */
    const double *alpha;         /* device [n_cells], turbulence parameter */
    const double *R;             /* device [n_cells], cylindrical radius, cm */
    const double *Z;             /* device [n_cells], height, cm */
    const double *eta;           /* device [n_cells] drift parameter, or NULL:
                                    no radial/azimuthal drift */
    const double *v_dust;        /* device [3][n_cells][N] (v_R, v_phi, v_Z) dust
                                    velocities, or NULL: terminal velocities from
                                    St, eta and Z */
    double v_frag;               /* fragmentation velocity, cm/s */
    double eta_frag;             /* fragment power law n(m) ~ m^-eta (11/6) */
    double chi_im;               /* impactor excavation factor (1) */
    double rho_m;                /* grain material density (1.6) */
    double mu;                   /* mean molecular weight (2.4) */
    double Mstar;                /* stellar mass, g */
    double k_B, m_H, G, sigma_H2;/* constants; sigma_H2 sets nu_mol */
    double kernel_const;         /* for CONSTANT / ADDITIVE kernels */
    int kernel_mode;             /* cudisc_kernel_mode */
    int frag_mode;               /* cudisc_frag_mode */
    int split_mode;              /* cudisc_split_mode */
    int precision;               /* cudisc_precision */
    double rtol;                 /* relative tolerance (1e-2) */
    double atol_rel;             /* absolute tolerance / sum_k rho_k (1e-10) */
    long long max_substeps;      /* per cell, accepted + rejected attempts */
    void *stream;                /* cudaStream_t, NULL = legacy default stream */
    int mixed_cluster;           /* CUDISC_MIXED_TF32 only: CTAs (one cluster) per
                                    group of 64 cell slots, 1, 2, 4 or 8, each
                                    taking that share of the contraction; 0 =
                                    chosen from n_cells and n_bins (see
                                    cudisc_coag_mixed_cluster).  A size whose
                                    buffers do not fit falls back to the
                                    largest smaller one that does. */
    int max_sms;                 /* SMs the integration kernels may occupy at
                                    once (their persistent grids are sized
                                    to it), so that several contexts run
                                    side by side; 0 = all.  The batched
                                    interface below sets it per disc. */
    int vertical;                /* 0: volume densities of (R, Z) cells (Sec. 5);
                                    1: vertically integrated kernel (Sec. 5.1):
                                    rho holds dust SURFACE densities per bin,
                                    each cell is a radius (Z unused), rho_gas
                                    its mid-plane gas density; grains form
                                    Gaussian layers of scale height
                                    h = H sqrt(alpha / (alpha + St)) (H =
                                    c_s / Omega_K), settle at their terminal
                                    velocity at Z = h (unless v_dust is given)
                                    and K_ij is divided by
                                    sqrt(2 pi (h_i^2 + h_j^2)).  The adjoint
                                    (cudisc_coag_vjp) differentiates h, the
                                    settling and that factor too. */
    int mixed_pair;              /* CUDISC_MIXED_TF32 only: 2 = CTA pairs share
                                    each M = 256 tensor-core MMA (tcgen05
                                    cta_group::2): a cluster of 2 x
                                    mixed_cluster CTAs serves two groups of 64
                                    slots, each CTA keeping half of every
                                    mapping tile (bins up to 128; else, or if it
                                    does not fit, single CTAs); 1 = single CTAs;
                                    0 = chosen at init (see
                                    cudisc_coag_mixed_pair). */
    int mixed_tile_stages;       /* CUDISC_MIXED_TF32 only: depth of the
                                    shared-memory ring of mapping tiles, in
                                    stages of two 16-pair blocks (1..4; 1 only
                                    with one CTA per group; CTA pairs 2..8);
                                    0 = chosen at init */
    int mixed_k_stages;          /* CUDISC_MIXED_TF32 only: depth of the
                                    shared-memory ring of the slots' K tables
                                    (1..4); 0 = chosen at init.  With either
                                    ring given, the rings take shared memory
                                    first and the per-slot integrator state
                                    follows only if it still fits (else it
                                    lives in the context's device workspace);
                                    cudisc_coag_init returns CUDISC_EINVAL
                                    when no cluster size takes the rings.
                                    The results do not depend on either
                                    depth, only the speed. */
    int cost_order;              /* 0 = the integration kernels (both
                                    precisions) hand cells to their slots in
                                    order of each cell's cost (accepted +
                                    rejected substeps) in the context's
                                    previous full-grid step, costliest first,
                                    which shortens the tail of a launch; the
                                    first step takes index order; 1 = always
                                    index order.  A cell's result does not
                                    depend on its slot, so the results are the
                                    same either way. */
} cudisc_coag_params;

typedef struct {
    long long accepted;          /* accepted substeps summed over cells */
    long long rejected;          /* rejected attempts summed over cells */
    long long max_accepted;      /* largest per-cell accepted count */
    int n_failed;                /* cells whose status is not CUDISC_OK */
    int worst_status;            /* largest per-cell status code */
    double mass_err_max;         /* max_c |sum_k rho'_ck / sum_k rho_ck - 1| */
    double elapsed_ms;           /* device time of the integration kernel */
} cudisc_step_stats;

/* Create a context: validates params (EINVAL on any inconsistency, naming the
 * field), builds the mapping tensors of Eqs. (Cijk), (Rijk), (fragrem) and
 * (Nijk) on the host in FP64, uploads them, allocates the workspace (and a
 * pinned host block of ~40 bytes per cell, into which each step's per-cell
 * results are read back), and builds K and p_frag from the gas arrays (as
 * cudisc_coag_build_kernel).
 * The device pointers in params must stay valid for the context's life. */
cudisc_status cudisc_coag_init(const cudisc_coag_params *params, cudisc_coag_ctx **out);

/* Rebuild the per-cell collision kernel K_ij and K_ij p_frag,ij (Sec. 5,
 * Eqs. kernel, vbrown, OCVrel, p_frag) from the current contents of the gas
 * arrays named at init (call after the caller changes them). */
cudisc_status cudisc_coag_build_kernel(cudisc_coag_ctx *ctx);

/* The same rebuild, only issued on the stream: no synchronisation and no
 * timing (cudisc_coag_get_timings keeps the last synchronous build's), so
 * that it may be captured in a CUDA graph together with
 * cudisc_coag_step_async. */
cudisc_status cudisc_coag_build_kernel_async(cudisc_coag_ctx *ctx);

/* Set the fragmentation velocity v_frag (cm/s, > 0 and finite, else
 * CUDISC_EINVAL).  Takes effect at the next cudisc_coag_build_kernel. */
cudisc_status cudisc_coag_set_v_frag(cudisc_coag_ctx *ctx, double v_frag);

/* Copy the kernel tables out for inspection: K_out and KF_out are device
 * [n_cells][Np] FP64, pair p = i (i + 1) / 2 + j for j <= i, holding K_ij and
 * K_ij p_frag,ij as stored by the context (mixed precision: the FP32
 * tables {K p_coag, K p_frag} widened, K = K p_coag + K p_frag in FP64). */
cudisc_status cudisc_coag_get_kernel(cudisc_coag_ctx *ctx, double *K_out, double *KF_out);

/* Right-hand side of Eq. (smol): drho_dt[c][k] for the state rho[c][k]
 * (device, [n_cells][N], FP64 in and out).  Asynchronous on the stream. */
cudisc_status cudisc_coag_rhs(cudisc_coag_ctx *ctx, const double *rho, double *drho_dt);

/* Integrate every cell over t_span seconds with BS3 3(2) (Sec. 5).
 * rho (device [n_cells][N]) is read and overwritten with the result.
 * dt_cell (device [n_cells], FP64, may be NULL): on entry the first step per
 * cell (<= 0: automatic), on exit the last proposed step.  stats (host, may
 * be NULL) receives totals.  Returns the worst per-cell status. */
cudisc_status cudisc_coag_step(cudisc_coag_ctx *ctx, double *rho, double t_span,
                               double *dt_cell, cudisc_step_stats *stats);

/* The same integration split in two: cudisc_coag_step_async only issues the
 * work on the stream (no host synchronisation, no allocation: it may be
 * captured in a CUDA graph and replayed); cudisc_coag_step_wait then
 * synchronises the stream, reads the per-cell results and fills stats (host,
 * may be NULL) for the last integration issued.  Arguments and statuses as
 * for cudisc_coag_step. */
cudisc_status cudisc_coag_step_async(cudisc_coag_ctx *ctx, double *rho, double t_span, double *dt_cell);
cudisc_status cudisc_coag_step_wait(cudisc_coag_ctx *ctx, cudisc_step_stats *stats);

/* As cudisc_coag_step with a span per cell: cell c is integrated over
 * t_span[c] seconds (device [n_cells], FP64).  A cell with t_span[c] <= 0
 * (or NaN) is left as it is: no steps, status OK, its rho and dt_cell
 * unchanged.  The cells to integrate are gathered on the device, so the
 * integration kernel's queue holds only those cells.  t_span NULL:
 * CUDISC_EINVAL.  Synchronises the stream. */
cudisc_status cudisc_coag_step_spans(cudisc_coag_ctx *ctx, double *rho, const double *t_span,
                                     double *dt_cell, cudisc_step_stats *stats);

/* Gas density from hydrostatic equilibrium (Sec. 3.5, Eqs. hydroeqbm,
 * hedisc, avcs, heprod, rhonorm), the rho_gas a context's kernel build
 * reads.  Per column i of an (R, Z) grid, for cells j = 0 .. n_Z - 1 in
 * order of height: P_j / P_{j-1} = exp[GM <1/c_s^2> (1/r_j - 1/r_{j-1})]
 * with <1/c_s^2> the mean of the two cells' 1/c_s^2, c_s^2 = k_B T /
 * (mu m_H), r = sqrt(R^2 + Z^2); P_j / P_0 their running product; the
 * density P / c_s^2 scaled so that sum_j rho_j V_j = Sigma_g,i (R dR)_i,
 * (R dR)_i = ((R_edges[i+1])^2 - R_edges[i]^2) / 2.
 * Device arrays, FP64, cell (i, j) at i * n_Z + j: R, Z (cell centres, cm),
 * T (K, > 0), V (cell volumes per radian, > 0), rho_gas (out, g cm^-3);
 * R_edges [n_R + 1] (cm), Sigma_g [n_R] (the column mass per unit area
 * held by its cells, g cm^-2).  mu, m_H (g), k_B (erg/K) and GM = G M_*
 * (cm^3 s^-2) must be positive.  Asynchronous on stream (a cudaStream_t,
 * NULL: the legacy default stream); allocates nothing; needs no context.
 * Errors: CUDISC_EINVAL for sizes < 1, NULL arrays or non-positive
 * constants (cudisc_coag_last_error(NULL) names it), CUDISC_ECUDA for a
 * failed launch. */
cudisc_status cudisc_hse_rho_gas(int n_R, int n_Z, const double *R, const double *Z, const double *T,
                                 const double *V, const double *R_edges, const double *Sigma_g, double mu,
                                 double m_H, double k_B, double GM, double *rho_gas, void *stream);

/* The source update of the dust dynamics step (Sec. 3.1, the full step's
 * items ii-iv with h = dt/2 and vi-viii with h = dt), for n_species dust
 * fluids on n_cells cells.  Conserved Q and primitive P_n are device
 * [4][n_species][n_cells] FP64: Q = (rho, rho v_R, rho v_phi R, rho v_Z)
 * after the transport (in; out: after the sources and drag), P_n = (rho,
 * v_R, v_phi, v_Z) at the start of the step.  Per cell (device [n_cells]):
 * R, Z (cm), rho_g (g cm^-3), c_s (cm/s); v_g device [3][n_cells] the gas
 * velocity (R, phi, Z); a device [n_species] grain radii (cm).  Steps:
 * Q += h (0, rho v_phi^2 / R - rho Omega^2 R, 0, -rho Omega^2 Z) on P_n
 * (Eq. sources without drag), Omega^2 = GM / (R^2 + Z^2)^(3/2); conversion
 * to primitives; the implicit drag v <- v - h / (h + t_s) (v - v_g) with
 * the Epstein t_s = rho_m a / (rho_g sqrt(8/pi) c_s) (Eqs. dragforce,
 * t_stop); back to conserved quantities.  rho must be positive.
 * Asynchronous on stream; allocates nothing; needs no context.  Errors:
 * CUDISC_EINVAL (sizes, NULL arrays, h < 0, rho_m <= 0, GM < 0),
 * CUDISC_ECUDA. */
cudisc_status cudisc_dust_source_update(int n_species, int n_cells, double *Q, const double *P_n, double h,
                                        const double *R, const double *Z, const double *rho_g,
                                        const double *c_s, const double *v_g, const double *a, double rho_m,
                                        double GM, void *stream);

/* The CFL time step of the dust dynamics (Sec. 3.1, Eqs. dtCFL, dt_adv,
 * dt_diff): the minimum over cells and species of C_adv |dR / v_R|,
 * C_adv |dZ / v_Z| (zero velocities impose none) and C_diff d^2 Sc / nu for
 * d = dR, dZ.  P device [4][n_species][n_cells] primitives (components 1
 * and 3 are read), dR, dZ, nu device [n_cells] (cm, cm, cm^2/s), Sc device
 * [n_species] Schmidt numbers; the paper's defaults are C_adv = 0.4 and
 * C_diff = 0.2.  dt_out is device FP64 [3]: the result in dt_out[0], the
 * largest |v| / d and the smallest Sc d^2 / nu in dt_out[1], dt_out[2]
 * (the reduction's workspace).  Inputs must be finite, with Sc, dR and dZ
 * positive and nu >= 0: a non-finite velocity, or an Sc, dR, dZ or nu
 * outside that range, makes dt_out[0] and dt_out[1] NaN (checked on the
 * device, so it shows when the caller reads the result).  Asynchronous on
 * stream; allocates nothing; calls that overlap on one dt_out race.  Errors
 * as above. */
cudisc_status cudisc_dust_cfl_dt(int n_species, int n_cells, const double *P, const double *dR, const double *dZ,
                                 const double *nu, const double *Sc, double C_adv, double C_diff, double *dt_out,
                                 void *stream);

/* The dust transport step of Sec. 3.1-3.2 (Eqs. quants, dynfluxes,
 * advgen, advdisc, fluxarea, halftimestepupdate, roeav, riemann, diffflux,
 * Fdiffmom, fluxes, weights, vkl, normaldecomp, F_k; Appendix A) on the
 * (R, theta) grid of Sec. 2, for n_species pressureless dust fluids: the
 * full step's items i-viii.  Stage 1: donor-cell face states of the
 * primitives at t^n, the upwind flux of the pressureless Riemann problem by
 * the sign of the Roe-averaged normal velocity (0 where the two sides move
 * apart), plus the diffusive flux -(rho_g nu / Sc) grad(rho / rho_g)
 * through the non-orthogonal stencil of Wu, Gao & Dai as the paper applies
 * it (each momentum component carried by the diffusive mass flux from its
 * upwind face state), Q* = Q^n - dt/2 (FA)^n / V, then the half-step
 * source update.  Stage 2: piecewise-linear face states of the n + 1/2
 * primitives with the van Leer limiter generalised to non-uniform grids,
 * the same fluxes, Q = Q^n - dt (FA)^(n+1/2) / V, then the full-step source
 * update.  The sources (curvature, gravity, exact implicit Epstein drag) are
 * those of cudisc_dust_source_update.
 * Grid: radial edges R_e [n_R + 1] (cm, increasing, > 0) and polar-angle
 * edges th_e [n_Z + 1] (radians above the mid-plane, increasing, |th| < 1.5)
 * as host arrays; centres R_c [n_R], th_c [n_Z] (host, NULL: midpoints);
 * cell (i, j) has centre (R_c[i], R_c[i] tan th_c[j]) and index c = i n_Z + j.
 * Geometry: volumes V = d(R^3)/3 d(tan th), radial face areas
 * (R_e)^2 d(tan th) and polar face areas d(R^2)/2 / cos(th_e) (cylindrical,
 * per radian of azimuth), or the planar V = d(R^2)/2 d(tan th), R_e d(tan
 * th), dR / cos(th_e) (cartesian, the paper's test geometry).
 * Boundaries bc[4] (inner R, outer R, lower theta, upper theta): OUTFLOW
 * (two ghost layers copy the adjacent active cell), CLOSED (the same, with
 * no flux through the boundary face), ZERO (ghosts at the floor density at
 * rest); the paper's default is {OUTFLOW, OUTFLOW, CLOSED, OUTFLOW} with the
 * mid-plane at th_e[0] = 0.  Ghost cells mirror the widths of the boundary
 * cells.
 * Fields (device, FP64): rho_g, nu [n_R n_Z] (gas density, kinematic
 * viscosity; nu NULL: no diffusion), Sc [n_species] (with nu); sources (all
 * or none; c_s NULL: transport only): c_s [n_R n_Z], v_g [3][n_R n_Z], a
 * [n_species], rho_m, GM.  The context keeps these pointers and its own
 * workspace (about 10 x 4 n_species n_R n_Z doubles).  A cell with density
 * <= 0 has zero velocity. */
typedef struct cudisc_dust_ctx cudisc_dust_ctx;   /* opaque, owned by the library */
typedef enum { CUDISC_GEOM_CYLINDRICAL = 0, CUDISC_GEOM_CARTESIAN = 1 } cudisc_geometry;
typedef enum { CUDISC_BC_OUTFLOW = 0, CUDISC_BC_CLOSED = 1, CUDISC_BC_ZERO = 2 } cudisc_boundary;
typedef struct {
    int n_species, n_R, n_Z;
    const double *R_e, *th_e;    /* host [n_R + 1], [n_Z + 1] */
    const double *R_c, *th_c;    /* host [n_R], [n_Z], or NULL: midpoints */
    int geometry;                /* cudisc_geometry */
    int bc[4];                   /* cudisc_boundary: inner R, outer R, lower th, upper th */
    double floor;                /* density of ZERO ghost cells */
    const double *rho_g, *nu;    /* device [n_R n_Z]; nu NULL: no diffusion */
    const double *Sc;            /* device [n_species] Schmidt numbers (with nu) */
    const double *c_s, *v_g, *a; /* device [n_R n_Z], [3][n_R n_Z], [n_species]; c_s NULL: no sources */
    double rho_m, GM;            /* grain material density; G M_* (sources) */
    void *stream;                /* cudaStream_t, NULL: legacy default stream */
} cudisc_dust_params;
/* Validate (CUDISC_EINVAL naming the field, through
 * cudisc_coag_last_error(NULL)), build the geometry on the host, allocate the
 * workspace and the diffusion stencil (as cudisc_dust_update_gas). */
cudisc_status cudisc_dust_init(const cudisc_dust_params *params, cudisc_dust_ctx **out);
/* Recompute the diffusion stencil's coefficients and the cached reciprocals
 * of rho_g and Sc after the caller changed the rho_g, nu or Sc arrays
 * (asynchronous on the stream). */
cudisc_status cudisc_dust_update_gas(cudisc_dust_ctx *ctx);
/* One full step of dt seconds (>= 0, finite): Q [4][n_species][n_R n_Z]
 * device FP64 (rho, rho v_R, rho v_phi R, rho v_Z), read and overwritten.
 * Asynchronous on the stream; allocates nothing (graph-capturable); steps on
 * one context must not overlap.  The CFL step is cudisc_dust_cfl_dt's. */
cudisc_status cudisc_dust_step(cudisc_dust_ctx *ctx, double *Q, double dt);
/* Copy the geometry out (device FP64, each may be NULL): V [n_R n_Z], radial
 * face areas AR [(n_R + 1) n_Z] (face a at R_e[a], row j: a n_Z + j), polar
 * face areas AZ [n_R (n_Z + 1)] (cell row i, face b at th_e[b]: i (n_Z + 1)
 * + b).  Synchronises the stream. */
cudisc_status cudisc_dust_geometry(const cudisc_dust_ctx *ctx, double *V, double *AR, double *AZ);
void cudisc_dust_destroy(cudisc_dust_ctx *ctx);

/* Sub-cycled coagulation (Sec. 6): the coagulation solver takes its own
 * sub-steps inside the global time steps of the disc model, and a cell's
 * coagulation is brought up to date only once one (by default) of its last
 * sub-steps has elapsed in global time.  Call once per global step of
 * dt_global seconds (>= 0, finite).  The context keeps, per cell, the
 * global time elapsed since its last update (its pending time, 0 at init).
 * Each call adds dt_global to it; a cell whose pending time has reached
 * trigger (> 0; 1 is the default of Sec. 6) times its last sub-step
 * dt_cell[c], or that has none yet (dt_cell NULL or dt_cell[c] <= 0), is
 * integrated over its whole pending time, which then restarts at 0; the
 * others are left as in cudisc_coag_step_spans.  dt_cell (device
 * [n_cells], may be NULL) is read and written as in cudisc_coag_step.
 * Synchronises the stream. */
cudisc_status cudisc_coag_subcycle(cudisc_coag_ctx *ctx, double *rho, double dt_global, double trigger,
                                   double *dt_cell, cudisc_step_stats *stats);

/* Copy the cells' pending times into pending (device [n_cells] FP64; NULL:
 * no copy) and, with reset != 0, set them to 0 (e.g. after the caller has
 * brought every cell up to date itself).  Synchronises the stream. */
cudisc_status cudisc_coag_subcycle_pending(cudisc_coag_ctx *ctx, double *pending, int reset);

/* Batched discs: n_discs independent problems (each with its own grid, bin
 * count and gas), integrated side by side.  Each disc gets a context of its
 * own (params[i], with its stream and max_sms replaced: the batch owns one
 * stream per disc and shares the SMs out in proportion to n_cells x
 * n_bins^2), so that all discs' persistent kernels are resident together.
 * The paper runs one disc at a time; this serves parameter studies. */
typedef struct cudisc_coag_batch cudisc_coag_batch;   /* opaque, owned by the library */
cudisc_status cudisc_coag_init_batched(const cudisc_coag_params *params, int n_discs,
                                       cudisc_coag_batch **out);
/* The context of disc i (owned by the batch: rhs, records, replay, vjp,
 * get_kernel and set_v_frag work on it as on any context; its stream is the
 * batch's stream for that disc). */
cudisc_status cudisc_coag_batch_ctx(cudisc_coag_batch *batch, int i, cudisc_coag_ctx **ctx);
/* Rebuild every disc's kernel tables (cudisc_coag_build_kernel), side by side. */
cudisc_status cudisc_coag_batch_build_kernel(cudisc_coag_batch *batch);
/* Integrate every disc over t_span: rho[i], dt_cell[i] as for cudisc_coag_step
 * on disc i (dt_cell may be NULL, or hold NULLs); stats (host [n_discs], may
 * be NULL) per disc.  The discs' work waits for what is already queued on
 * stream (NULL: legacy default stream) and the call returns when all discs
 * are done.  Returns the worst status over the discs (their messages: the
 * discs' contexts).  The discs' persistent kernels run side by side only if
 * their streams have hardware queues of their own: CUDA maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS queues (8 by default, set in the environment
 * before CUDA initialises), and discs sharing a queue run one after another
 * (a 32-disc batch took 9.9 s per step instead of 4.2 s).  A CUDA graph of
 * cudisc_coag_batch_step_async runs them side by side either way. */
cudisc_status cudisc_coag_batch_step(cudisc_coag_batch *batch, double *const *rho, double t_span,
                                     double *const *dt_cell, void *stream, cudisc_step_stats *stats);
/* The same split in two, as cudisc_coag_step_async / _step_wait for one
 * disc: _async issues every disc's integration (no kernel rebuild) on the
 * disc's stream, forked from stream by an event and joined back to it, and
 * returns without synchronising or allocating, so that the whole batch is
 * one stretch of stream's work (a single CUDA graph when stream is being
 * captured; issue one cudisc_coag_batch_step first, outside the capture, so
 * that each disc's kernel attributes are set); _wait synchronises each disc
 * and writes stats (host [n_discs], may be NULL) for the last issue.  EINVAL
 * for NULL arguments or a bad t_span; a disc's launch error stops the issue
 * at that disc. */
cudisc_status cudisc_coag_batch_step_async(cudisc_coag_batch *batch, double *const *rho, double t_span,
                                           double *const *dt_cell, void *stream);
cudisc_status cudisc_coag_batch_step_wait(cudisc_coag_batch *batch, cudisc_step_stats *stats);
void cudisc_coag_batch_destroy(cudisc_coag_batch *batch);

/* Shards for several GPUs.  During a coagulation call every cell evolves on
 * its own (Sec. 2: the per-cell update; Sec. 5), so a job spreads over GPUs
 * with no exchange: each process takes a contiguous range of the cells (in
 * index order c = i_R n_Z + i_Z, so a range of radii) or of whole discs,
 * builds its own context on it (pointers offset to the range's first cell)
 * and integrates it.  This splits n_items consecutive items with costs cost
 * (host [n_items], finite, >= 0; NULL: 1 each; e.g. accepted substeps per
 * cell from an earlier step, or n_cells x N^2 per disc) into n_parts ranges
 * whose largest total cost is the smallest any contiguous split reaches
 * (to 1e-13 relative): range k is items bounds[k] .. bounds[k+1] - 1
 * (bounds host [n_parts + 1], bounds[0] = 0, bounds[n_parts] = n_items,
 * nondecreasing; trailing ranges may be empty).  Host only; needs no GPU
 * or context.  Errors: CUDISC_EINVAL for n_items < 0, n_parts < 1, a NULL
 * bounds or a negative or non-finite cost. */
cudisc_status cudisc_partition(int n_items, const double *cost, int n_parts, int *bounds);

/* Optional per-cell records for later cudisc_coag_step calls (all device
 * pointers; pass NULLs to stop recording):
 *   dt_log [n_cells][log_cap] accepted step sizes in order,
 *   n_log  [n_cells] int64 number of accepted steps (may exceed log_cap:
 *          only the first log_cap are stored),
 *   status [n_cells] int32 per-cell status. */
cudisc_status cudisc_coag_set_records(cudisc_coag_ctx *ctx, double *dt_log,
                                      long long log_cap, long long *n_log,
                                      int *status);

/* Fixed-step replay: apply per-cell sequences of BS3 steps without error
 * control (hs [n_cells][stride] device FP64, n_h [n_cells] device int64).
 * Used to compare precisions on one step sequence. */
cudisc_status cudisc_coag_replay(cudisc_coag_ctx *ctx, double *rho, const double *hs,
                                 const long long *n_h, long long stride);

/* Same integration as cudisc_coag_step on a CUDISC_MIXED_TF32 context, but
 * the per-cell-slot integrator scratch lives in a fixed 16 MiB device array
 * compiled into the library instead of the context's workspace.  The paper
 * has no counterpart: this is for callers that cannot allocate device memory
 * at the point where they integrate, for example a code whose device memory
 * is wholly owned by its own pool allocator, or a time loop that must not take
 * cudaMalloc's implicit device synchronisation.  This call itself allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine); the caller
 * passes rho and dt_cell exactly as for cudisc_coag_step.
 *   - The scratch holds the per-slot FP32 state (state pair and stage
 *     right-hand sides) when it does not fit in the kernel's shared memory;
 *     cudisc_coag_scratch_bytes gives its size for a context (0: shared
 *     memory holds it and the array is not touched).
 *   - The first call on each context looks up the array's device address
 *     (cudaGetSymbolAddress, with the context's device current); make that
 *     first call before any stream capture.
 *   - Every GPU that loads the library holds the 16 MiB until the process
 *     exits, whether or not this entry point is used.
 *   - All calls share the one array (it keeps the last call's contents, and
 *     every slot's state is written before it is read): calls that overlap
 *     on the GPU, from any context, race and give wrong results.
 *   - Problems whose scratch exceeds 16 MiB (slot groups x 64 slots x 5 x N x
 *     4 bytes when it is used; see cudisc_coag_mixed_cluster for the groups)
 *     are rejected with CUDISC_ENOTSUP and a message; use cudisc_coag_step
 *     for them.
 *   - Returns CUDISC_EINVAL for a context of another precision. */
cudisc_status cudisc_coag_step_static_scratch(cudisc_coag_ctx *ctx, double *rho, double t_span,
                                              double *dt_cell, cudisc_step_stats *stats);

/* The integration of cudisc_coag_step from and to HOST memory, for callers
 * whose state lives on the host: copies rho_in (host [n_cells][N], FP64) to
 * a device state array the context keeps, rebuilds the kernel tables from
 * the gas arrays when rebuild != 0 (as cudisc_coag_build_kernel), integrates
 * every cell over t_span with fresh initial step sizes (dt_cell NULL), and
 * copies the result to rho_out (host [n_cells][N]; may be rho_in).  All on
 * the context's stream, which is synchronised before the call returns,
 * except the copy-in when rebuild != 0: it runs on a second stream of the
 * context beside the table build (which reads the gas arrays only), forked
 * after the stream's earlier work and joined before the integration.
 *   - Pinned host memory (cudaHostAlloc / cudaHostRegister) makes both
 *     copies DMA transfers; pageable memory works, through the driver's
 *     staging buffers.
 *   - The device state array (n_cells x N doubles), the second stream and
 *     its two events are created at the first call on a context and freed
 *     by cudisc_coag_destroy; later calls allocate nothing.
 *   - stats as cudisc_coag_step (elapsed_ms: the integration alone).
 *   - CUDISC_EINVAL for a NULL context or host pointer; per-cell failures as
 *     cudisc_coag_step (rho_out then holds the states reached). */
cudisc_status cudisc_coag_step_host(cudisc_coag_ctx *ctx, const double *rho_in, double *rho_out, double t_span,
                                    int rebuild, cudisc_step_stats *stats);

/* Failure-path test hook of the mixed-precision integration kernel (the
 * paper has no counterpart).  Every wait of that kernel on another role's
 * progress is bounded by a clock limit (~2 s); when one runs out the kernel
 * records the fact in a status word, waits (with its own bound) for the
 * bulk copies and MMAs it has issued, frees its tensor memory and returns,
 * and the call reports CUDISC_ECUDA ("a bounded device wait ran out").
 * wait_cycles > 0 sets that limit in SM clocks for later integrations on
 * this context (0: the default); withhold = 1 makes the kernel's bulk-copy
 * producer issue no copies, so that every consumer's wait runs out (needs
 * wait_cycles > 0).  (0, 0) restores normal operation.  Host only;
 * CUDISC_EINVAL for other values.  FP64 contexts ignore it. */
cudisc_status cudisc_coag_set_fault_injection(cudisc_coag_ctx *ctx, long long wait_cycles, int withhold);

/* Bytes of device scratch beyond the context's tables that one integration
 * of the mixed-precision kernel uses for its per-slot state: slot groups x
 * 64 slots x 5 x N x 4 when that state does not fit in shared memory, else
 * 0 (also 0 for an FP64 context).  cudisc_coag_step takes it from the
 * context's workspace, cudisc_coag_step_static_scratch from its fixed
 * array.  EINVAL for a NULL argument.  Host only. */
cudisc_status cudisc_coag_scratch_bytes(const cudisc_coag_ctx *ctx, size_t *bytes);

/* Device times (CUDA events on params.stream) of the last call of each kind:
 * the per-cell prep and the kernel-table build of cudisc_coag_build_kernel,
 * the integration kernel of cudisc_coag_step (also in stats.elapsed_ms) and
 * the whole of cudisc_coag_vjp.  0 for a kind not yet called.  Host only. */
typedef struct {
    double prep_ms;
    double kbuild_ms;
    double step_ms;
    double vjp_ms;
} cudisc_timings;
cudisc_status cudisc_coag_get_timings(const cudisc_coag_ctx *ctx, cudisc_timings *out);

/* Launch layout of the mixed-precision integration kernel chosen at init:
 * *cluster = CTAs per group of 64 cell slots (1, 2, 4 or 8; the contraction
 * of a group's pass is split between them), *groups = groups resident at
 * once.  Both 0 for an FP64 context.  EINVAL for a NULL argument.  Host only. */
cudisc_status cudisc_coag_mixed_cluster(const cudisc_coag_ctx *ctx, int *cluster, int *groups);

/* *pair = 1 when the mixed-precision kernel of this context runs in CTA
 * pairs (see mixed_pair), else 0 (also for an FP64 context).  EINVAL for a
 * NULL argument.  Host only. */
cudisc_status cudisc_coag_mixed_pair(const cudisc_coag_ctx *ctx, int *pair);

/* Ring depths of the mixed-precision kernel of this context: *tile_stages
 * (mapping tiles) and *k_stages (K tables), in stages of two blocks, and
 * *state_in_smem = 1 when the per-slot integrator state is in shared memory
 * (0: in the device workspace).  All 0 for an FP64 context.  EINVAL for a
 * NULL argument.  Host only. */
cudisc_status cudisc_coag_mixed_rings(const cudisc_coag_ctx *ctx, int *tile_stages, int *k_stages,
                                      int *state_in_smem);

/* Vector-Jacobian product of the integration (the paper has no adjoint; this
 * is the discrete adjoint of the BS3 map of Sec. 5 with the step sizes held
 * fixed).  For L = sum_{c,k} grad_rhoT[c][k] rho_ck(T), where rho(T) is
 * reached from rho0 by a per-cell sequence of accepted BS3 steps, it writes
 *   grad_rho0  [n_cells][N] device FP64: dL / d rho0,
 *   grad_alpha [n_cells]    device FP64: dL / d alpha_c (through v_turb,
 *                           Re = nu_t / nu_mol and St*), or NULL,
 *   grad_vfrag [1]          device FP64: dL / d v_frag summed over cells
 *                           (through p_frag), or NULL.
 * The step sequence is either given (hs [n_cells][stride] device FP64,
 * n_h [n_cells] device int64, 0 <= n_h[c] <= stride: e.g. the records of a
 * cudisc_coag_step call, see cudisc_coag_set_records; t_span is ignored) or,
 * with hs == NULL, taken from a fresh adaptive integration of rho0 over
 * t_span with an automatic first step (n_h and stride ignored).  rho0 and
 * grad_rhoT are device [n_cells][N] FP64 and are not modified.
 * The adjoint runs one CTA per cell: a forward pass keeps the state every 16
 * substeps, and each 16-substep segment is recomputed before its reverse
 * sweep.  Arithmetic is FP64 for contexts of either precision (FP32 loses
 * the gradient with respect to large grains, a small difference of
 * sweep-up sums), or double-float for the per-pair work after
 * cudisc_coag_set_adjoint_precision; K and K p_frag are the context's current tables
 * (cudisc_coag_build_kernel), so a CUDISC_MIXED_TF32 context differentiates
 * its own map with FP32 kernel tables.  The context's
 * adjoint tables are built on the first call and its checkpoint storage
 * (n_cells x ceil(max n_h / 16) x N values) grows when a longer sequence
 * arrives; later calls of the same size allocate nothing.
 * Errors: CUDISC_EINVAL (NULL arrays, n_h outside [0, stride]),
 * CUDISC_ENOTSUP (N too large for the per-cell shared memory; every
 * N <= 160 fits), the forward's per-cell status when
 * hs == NULL and that integration fails, CUDISC_ENONFINITE when a cell's
 * gradient is not finite.  Synchronises the stream. */
cudisc_status cudisc_coag_vjp(cudisc_coag_ctx *ctx, const double *rho0, double t_span,
                              const double *hs, const long long *n_h, long long stride,
                              const double *grad_rhoT, double *grad_rho0, double *grad_alpha,
                              double *grad_vfrag);

/* Arithmetic of the per-pair work of later cudisc_coag_vjp calls on ctx
 * (the paper has no adjoint; see cudisc_coag_vjp): CUDISC_ADJOINT_FP64 (the
 * default) or CUDISC_ADJOINT_DOUBLE_FLOAT, in which the forward recompute's
 * right-hand sides and the transposed right-hand sides run in double-float
 * (each value an unevaluated sum of two FP32 numbers; error-free FP32 sums
 * and products), while the stage vectors, checkpoints and parameter-gradient
 * sums stay FP64.  B300 executes FP64 at a small fraction of its FP32 rate,
 * and the FP64 adjoint is bound by its FP64 pipe.  The FP32 exponent range
 * applies to the per-pair terms: products below ~1e-38 of the cell's dust
 * mass scale flush to zero.  The adjoint tables are rebuilt for the new type
 * at the next cudisc_coag_vjp.  EINVAL for another value or a NULL ctx.
 * Host only; allocates nothing. */
cudisc_status cudisc_coag_set_adjoint_precision(cudisc_coag_ctx *ctx, int precision);

void cudisc_coag_destroy(cudisc_coag_ctx *ctx);

/* Message of the last failed call on ctx (or of this thread when ctx is
 * NULL); never NULL, "" when there was no error. */
const char *cudisc_coag_last_error(const cudisc_coag_ctx *ctx);

/* Library version string. */
const char *cudisc_coag_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CUDISC_COAG_H */
