// Internal declarations of the B300 coagulation library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cudisc_coag.h"

namespace cdc {

struct VjpState;                      // adjoint tables and workspace (vjp.cu)

constexpr int kMaxBins = 160;         // FP64 path keeps the pair weights of one cell in smem
constexpr int kBlkPairs = 16;         // pairs per K-block of the mixed contraction
constexpr int kBlkElems = 32;         // TF32 elements per K-block row (a and b per pair)
constexpr int kMaxMixedBins = 160;    // mixed path: bins up to this (MMA N = bins rounded up to 16)
constexpr int kMaxGridY = 65535;      // launches over cells are chunked to this

// Layout of the mixed path's FP32 kernel tables {K p_coag, K p_frag}:
// cell-major, n_slots = 16 n_blk pair slots per cell (pair slot q = 16 b + t
// of block b), so a cell's table is 8 n_slots contiguous bytes.  The
// integration kernel copies the table of each cell it takes into its slot
// group's buffer (see the mixed kernel).
__host__ __device__ inline size_t k32_index(int c, int q, int n_slots) { return (size_t)c * n_slots + q; }

// Rows of each mapping tile of the mixed contraction (the bins, padded):
// up to 128 bins the hi and lo tiles form one MMA operand of N = 2 NBP,
// which needs NBP to be a multiple of 8; above, each is its own operand of
// N = NBP, a multiple of 16.
inline int mixed_nbp(int N)
{
    const int n8 = (N + 7) / 8 * 8;
    return 2 * n8 <= 256 ? n8 : (N + 15) / 16 * 16;
}

// Per-cell scalars produced by the prep kernel (FP64).
struct CellScal {
    double kT8pi;   // 8 k_B T / pi  (Eq. vbrown numerator per unit mass sum)
    double Vg2;     // alpha c_s^2   (eddy velocity squared)
    double delta;   // Re^-1/2       (Kolmogorov Stokes number)
    double etavK;   // eta Omega R   (drift velocity scale)
    double ZOm;     // Z Omega       (settling velocity scale)
    double pad;
};

// Per-cell, per-bin fields of the prep kernel, stored [cell][field][N].
// PF_H: grain scale height (vertically integrated kernel; 0 otherwise).
enum PrepField { PF_ST = 0, PF_VR, PF_VPHI, PF_VZ, PF_G1, PF_G2, PF_H, PF_COUNT };
// FP32 copy: St and each input velocity as an FP32 hi/lo pair, so that
// differences of nearly equal velocities keep their precision.
// P3_SS, P3_SSMD, P3_OMSS: St* = clamp(1.6 St, Re^-1/2, 1), St* - Re^-1/2 and
// 1 - St* of the bin when it is the larger of a pair, formed in FP64 (both
// differences can be tiny next to their operands).
// P3_U = 8 k_B T / (pi m_k) (so v_BM^2 = U_i + U_j), P3_A = a_k, P3_M = m_k:
// the pair loop of the FP32 builder then needs no FP64 arithmetic.
// P3_HH = 2 pi h^2 (vertically integrated kernel: K / sqrt(HH_i + HH_j)).
enum Prep32Field { P3_ST = 0, P3_VRH, P3_VRL, P3_VPH, P3_VPL, P3_VZH, P3_VZL,
                   P3_SS, P3_SSMD, P3_OMSS, P3_U, P3_A, P3_M, P3_HH, P3_COUNT };

// Per-cell integration scalars written back by the step kernels.
struct CellOut {
    long long n_acc, n_rej;
    double h_last;
    double mass_err;
    int status;
    int pad;
};

// Launch-time view of the tables the kernels read (all device pointers).
struct DevTables {
    int N, Np, n_cells;
    const double *m, *minv, *a, *me;          // [N], me [N+1]
    const unsigned int *pair_ij;              // [Np] (i << 16) | j
    // FP64 gather form of Eq. (smol): per output bin k, entries (p, alpha, beta)
    const int *row;                           // [N+1]
    const int *ent_p;                         // [nnz]
    const double2 *ent_ab;                    // [nnz]
    const int *frow;                          // [N+1] fragment gather per bin l
    const int *fent_p;                        // [fnnz]
    const double *fent_m;                     // [fnnz]
    const double *Ntab;                       // [N][N] row l, col k: N_k(m^e_{l+1})
    // mixed path
    int n_blk;
    const int *blk_i, *blk_j0;                // [n_blk]
    const float4 *Btiles;                     // [n_blk][2][NBP][32] swizzled TF32 hi/lo, NBP = N rounded to 16
};

} // namespace cdc

struct cudisc_coag_ctx {
    cudisc_coag_params p;
    cudaStream_t stream = nullptr;
    int N = 0, Np = 0, n_cells = 0, n_blk = 0;
    std::string err;
    // host copies
    std::vector<double> h_m, h_me;
    // device tables
    double *d_m = nullptr, *d_minv = nullptr, *d_a = nullptr, *d_me = nullptr;
    unsigned int *d_pair_ij = nullptr;
    int *d_row = nullptr, *d_ent_p = nullptr, *d_frow = nullptr, *d_fent_p = nullptr;
    double2 *d_ent_ab = nullptr;
    double *d_fent_m = nullptr, *d_Ntab = nullptr;
    int *d_blk_i = nullptr, *d_blk_j0 = nullptr;
    float4 *d_Btiles = nullptr;
    // per-cell prep and kernel tables
    double *d_prep = nullptr;          // [n_cells][PF_COUNT][N]
    float *d_prep32 = nullptr;         // same, FP32
    cdc::CellScal *d_scal = nullptr;   // [n_cells]
    float4 *d_scal32 = nullptr;        // [n_cells] {delta, Vg2, etavK, ZOm} in FP32
    double2 *d_K64 = nullptr;          // [n_cells][Np]      {K, K p_frag}
    float2 *d_K32 = nullptr;           // n_cells x n_blk x 16 {K p_coag, K p_frag}, see k32_index
    float4 *d_Kslot = nullptr;         // mixed kernel: [group][block][8 chunks][64 slots] of the slots' tables
    int mix_P = 1, mix_G = 1, mix_C = 1;   // mixed kernel: CTAs per slot group, groups, initial cells per group
    int mix_pair = 0;                  // mixed kernel: CTA pairs share M = 256 MMAs
    bool timed = false;                // the last integration issued recorded ev0/ev1
    void *static_scratch = nullptr;    // device address of the fixed scratch array (first static call)
    double *d_host_state = nullptr;    // [n_cells][N] device state of cudisc_coag_step_host (first call)
    cudaStream_t copy_stream = nullptr;   // cudisc_coag_step_host: the state's copy-in beside the kernel build
    cudaEvent_t ev_fork = nullptr, ev_copied = nullptr;
    void *h_stats = nullptr;           // pinned: the status word, then [n_cells] CellOut (finish_step's reads)
    long long inject_wait_cycles = 0;  // test hook: wait limit of the mixed kernel (0: the default)
    int inject_withhold = 0;           // test hook: the mixed kernel's producer issues no copies
    // integration workspace
    cdc::CellOut *d_out = nullptr;     // [n_cells]
    double *d_work = nullptr;          // mixed path slot state
    size_t work_bytes = 0;
    int *d_counter = nullptr;          // work queue head (d_counter[3]: work-list length)
    int *d_list = nullptr;             // [n_cells] work list of per-cell-span integrations
    int *d_order = nullptr;            // [n_cells] cells by the previous full-grid step's cost (identity at first)
    double *d_spans = nullptr;         // [n_cells] their spans
    double *d_pending = nullptr;       // [n_cells] global time since each cell's last sub-cycled update
    // optional records
    double *rec_dt = nullptr; long long rec_cap = 0; long long *rec_n = nullptr;
    int *rec_status = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evb[3] = {nullptr, nullptr, nullptr};   // prep | kbuild | end
    double t_prep = 0.0, t_kbuild = 0.0, t_step = 0.0, t_vjp = 0.0;   // ms, last call
    cdc::VjpState *vjp = nullptr;      // built on the first cudisc_coag_vjp
    int adj_prec = CUDISC_ADJOINT_FP64;   // arithmetic of cudisc_coag_vjp's per-pair work

    cdc::DevTables tables() const;
};

namespace cdc {
// The cells an integration covers: all of them (cells == NULL) or
// cells[0 .. *count - 1] (device; the count is read by the kernels), each
// over spans[c] seconds (device [n_cells]; NULL: the call's t_span).
struct WorkList {
    const int *cells = nullptr;
    const int *count = nullptr;
    const double *spans = nullptr;
};
// kernel launchers (defined in the .cu files)
cudaError_t launch_prep(const cudisc_coag_ctx *c);
cudaError_t launch_kbuild(const cudisc_coag_ctx *c);
cudaError_t launch_get_kernel(const cudisc_coag_ctx *c, double *K, double *KF);
cudaError_t launch_rhs_fp64(const cudisc_coag_ctx *c, const double *rho, double *drho);
cudaError_t launch_step_fp64(const cudisc_coag_ctx *c, double *rho, double t_span,
                             double *dt_cell, const double *replay_h,
                             const long long *replay_n, long long replay_stride, WorkList wl = WorkList());
cudaError_t launch_rhs_mixed(const cudisc_coag_ctx *c, const double *rho, double *drho);
cudaError_t launch_step_mixed(const cudisc_coag_ctx *c, double *rho, double t_span,
                              double *dt_cell, const double *replay_h,
                              const long long *replay_n, long long replay_stride, WorkList wl = WorkList());
size_t mixed_workspace_bytes(int n_cells, int N, int P, int max_sms, int pair, int sb_req, int ks_req);
// CTAs per slot group P for a request P_req (0: automatic), groups of slots G,
// initial cells per group C and CTA-pair mode (pair_req: 0 automatic, 1 off,
// 2 on) of the mixed kernel
bool mixed_layout(int n_cells, int N, int P_req, int max_sms, int pair_req, int sb_req, int ks_req, int *P, int *G,
                  int *C, int *pair);
void mixed_rings(int n_cells, int N, int P, int max_sms, int pair, int sb_req, int ks_req, int *SB, int *KS,
                 int *state_smem);
// hydrostatic-equilibrium gas density (hse.cu)
cudaError_t launch_hse(int n_R, int n_Z, const double *R, const double *Z, const double *T, const double *V,
                       const double *R_edges, const double *Sigma_g, double mu, double m_H, double k_B,
                       double GM, double *rho, cudaStream_t stream);
// dust source update and CFL step (dust.cu)
cudaError_t launch_dust_source(int n_s, int n_c, double *Q, const double *Pn, double h, const double *R,
                               const double *Z, const double *rho_g, const double *c_s, const double *v_g,
                               const double *a, double rho_m, double GM, cudaStream_t stream);
cudaError_t launch_dust_cfl(int n_s, int n_c, const double *P, const double *dR, const double *dZ,
                            const double *nu, const double *Sc, double C_adv, double C_diff, double *dt,
                            cudaStream_t stream);
// adjoint (vjp.cu)
bool vjp_fits(const cudisc_coag_ctx *c);
cudaError_t vjp_prepare(cudisc_coag_ctx *c, long long max_steps);
cudaError_t vjp_records(cudisc_coag_ctx *c, long long cap, double **dt, long long **n, int **status,
                        double **rho_tmp);
cudaError_t launch_vjp(cudisc_coag_ctx *c, const double *rho0, const double *hs,
                       const long long *n_h, long long stride, const double *w, double *g_rho0,
                       double *g_alpha, double *g_vf);
cudaError_t vjp_worst_status(const cudisc_coag_ctx *c, int *worst);
void vjp_free(cudisc_coag_ctx *c);
// the thread's last error message (cudisc_coag_last_error(NULL)), for entry
// points outside coag_host.cu
void set_thread_error(const std::string &msg);
// fixed-scratch variant of the mixed step (see cudisc_coag_step_static_scratch)
size_t static_scratch_bytes();
cudaError_t launch_step_mixed_static(cudisc_coag_ctx *c, double *rho, double t_span,
                                     double *dt_cell, bool *too_big);
// bytes of global scratch the mixed integration's per-slot state takes (0:
// it is kept in shared memory)
size_t mixed_scratch_bytes(int n_cells, int N, int P, int max_sms, int pair, int sb_req, int ks_req);
} // namespace cdc
