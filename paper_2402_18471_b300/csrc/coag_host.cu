// Host side of the C ABI: validation, the FP64 mapping-tensor builder
// (Sec. 5, Eqs. Cijk, Rijk, fragrem, fragdist, Nijk), device tables and the
// dispatch to the FP64 and mixed-precision kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "coag_internal.h"

using cdc::CellOut;

namespace {

thread_local std::string g_thread_err;
// byte offset of the per-cell results in a context's pinned read-back block
// (the status word comes first)
constexpr size_t kStatsOff = 64;

} // namespace

void cdc::set_thread_error(const std::string &msg) { g_thread_err = msg; }

namespace {

cudisc_status fail(cudisc_coag_ctx *c, cudisc_status st, const std::string &msg)
{
    if (c) c->err = msg;
    g_thread_err = msg;
    return st;
}

cudisc_status cuda_fail(cudisc_coag_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    cudisc_status st = (e == cudaErrorMemoryAllocation) ? CUDISC_ENOMEM : CUDISC_ECUDA;
    return fail(c, st, m);
}

#define CUDA_TRY(ctx, expr)                                   \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

// Work list of an integration with per-cell spans: cells with a positive
// span (given, or, sub-cycling, the pending global time once it reaches
// trigger x the cell's last sub-step) are listed; the others get an empty
// result record (no steps, status OK, their state and dt_cell kept).
// The order in which the next full-grid step hands cells to its slots:
// costliest first by this step's accepted + rejected substeps, in buckets of
// 1/16 octave (counting sort in one CTA; the order within a bucket is
// whatever the atomics give, which is harmless because a cell's result does
// not depend on its slot).
constexpr int kOrderBuckets = 256;
__device__ __forceinline__ int cost_bucket(const CellOut &o)
{
    const long long cost = o.n_acc + o.n_rej;
    if (cost <= 0) return 0;
    const int b = 1 + (int)(16.0f * __log2f((float)cost));
    return b < kOrderBuckets - 1 ? b : kOrderBuckets - 1;
}

__global__ void __launch_bounds__(1024) cost_order_kernel(int n_cells, const CellOut *__restrict__ out,
                                                          int *__restrict__ order)
{
    __shared__ int hist[kOrderBuckets], base[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < n_cells; c += blockDim.x) atomicAdd(&hist[cost_bucket(out[c])], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int sum = 0;
        for (int b = kOrderBuckets - 1; b >= 0; b--) { base[b] = sum; sum += hist[b]; }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n_cells; c += blockDim.x) order[atomicAdd(&base[cost_bucket(out[c])], 1)] = c;
}

__global__ void iota_kernel(int n, int *v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

__global__ void worklist_kernel(int n_cells, const double *span_in, double *pending, double dt_global,
                                double trigger, const double *dt_cell, double *spans, int *list, int *count,
                                CellOut *out, long long *rec_n, int *rec_status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    double span;
    if (span_in) {
        span = span_in[c];
    } else {
        const double acc = pending[c] + dt_global;
        const double h = dt_cell ? dt_cell[c] : 0.0;
        const bool due = !(h > 0.0) || acc >= trigger * h;
        span = due ? acc : 0.0;
        pending[c] = due ? 0.0 : acc;
    }
    if (span > 0.0) {
        spans[c] = span;
        list[atomicAdd(count, 1)] = c;
    } else {
        CellOut o;
        o.n_acc = 0;
        o.n_rej = 0;
        o.h_last = dt_cell ? dt_cell[c] : 0.0;
        o.mass_err = 0.0;
        o.status = CUDISC_OK;
        o.pad = 0;
        out[c] = o;
        if (rec_n) rec_n[c] = 0;
        if (rec_status) rec_status[c] = CUDISC_OK;
    }
}

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &src, cudaStream_t s)
{
    size_t n = src.size() ? src.size() : 1;
    cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
    if (e != cudaSuccess) return e;
    if (src.empty()) return cudaSuccess;
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// Mass fraction of fragments in bin k when the largest fragment fills bin l:
// integral of m n(m) dm with n ~ m^-eta over bin k, normalised over bins 0..l.
double frag_share(const std::vector<double> &me, double eta, int k, int l)
{
    double s = 2.0 - eta;
    if (std::fabs(s) < 1e-12)
        return std::log(me[k + 1] / me[k]) / std::log(me[l + 1] / me[0]);
    double lo = std::pow(me[0], s);
    return (std::pow(me[k + 1], s) - std::pow(me[k], s)) / (std::pow(me[l + 1], s) - lo);
}

// Round an FP32 value to the nearest TF32 value (ties to even).
uint32_t tf32_rn_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return u & 0xFFFFE000u;
    u += 0xFFFu + ((u >> 13) & 1u);
    return u & 0xFFFFE000u;
}

float bits_f(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }

// Double-double arithmetic (error-free transforms: Knuth's TwoSum and the
// FMA form of Dekker's TwoProduct).  A pair whose grains differ in mass by
// up to 1e21 adds and removes m_i-sized masses at bin i while moving only
// an m_j-sized mass; summing those terms in plain FP64 leaves an error of
// ~1e-16 m_i, which can exceed the transfer itself.  Accumulating each net
// coefficient in double-double makes every pair conserve mass to the
// rounding of its own transfer.
struct dd { double hi, lo; };
dd dd_of(double a) { return {a, 0.0}; }
dd two_sum(double a, double b)
{
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
dd fast_two_sum(double a, double b) { double s = a + b; return {s, b - (s - a)}; }
dd operator+(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
dd operator-(dd a) { return {-a.hi, -a.lo}; }
dd operator-(dd a, dd b) { return a + (-b); }
dd operator*(dd a, dd b)
{
    double p = a.hi * b.hi;
    double e = std::fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p, e);
}
dd operator/(dd a, dd b)
{
    double q1 = a.hi / b.hi;
    dd r = a - b * dd_of(q1);
    double q2 = r.hi / b.hi;
    r = r - b * dd_of(q2);
    double q3 = r.hi / b.hi;
    return fast_two_sum(q1, q2) + dd_of(q3);
}
double dd_val(dd a) { return a.hi + a.lo; }

// two_bin in double-double: the mass fractions of the lower and upper bin.
void two_bin_dd(const std::vector<double> &m, dd mass, int mode, int &kl, int &ku, dd &fl, dd &fu)
{
    const int N = (int)m.size();
    if (dd_val(mass - dd_of(m[N - 1])) >= 0.0) { kl = ku = N - 1; fl = dd_of(1.0); fu = dd_of(0.0); return; }
    if (dd_val(mass - dd_of(m[0])) <= 0.0) { kl = ku = 0; fl = dd_of(1.0); fu = dd_of(0.0); return; }
    int lo = 0, hi = N - 1;               // m[lo] <= mass < m[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (dd_val(mass - dd_of(m[mid])) >= 0.0) lo = mid; else hi = mid;
    }
    kl = lo; ku = lo + 1;
    const dd span = dd_of(m[ku]) - dd_of(m[kl]);
    const dd up = (mass - dd_of(m[kl])) / span;          // 1 - eps
    const dd eps = (dd_of(m[ku]) - mass) / span;
    if (mode == CUDISC_SPLIT_NUMBER) {
        fl = eps * dd_of(m[kl]) / mass;
        fu = up * dd_of(m[ku]) / mass;
    } else {
        fl = eps;
        fu = up;
    }
}

} // namespace

cdc::DevTables cudisc_coag_ctx::tables() const
{
    cdc::DevTables t;
    t.N = N; t.Np = Np; t.n_cells = n_cells;
    t.m = d_m; t.minv = d_minv; t.a = d_a; t.me = d_me;
    t.pair_ij = d_pair_ij;
    t.row = d_row; t.ent_p = d_ent_p; t.ent_ab = d_ent_ab;
    t.frow = d_frow; t.fent_p = d_fent_p; t.fent_m = d_fent_m;
    t.Ntab = d_Ntab;
    t.n_blk = n_blk; t.blk_i = d_blk_i; t.blk_j0 = d_blk_j0;
    t.Btiles = d_Btiles;
    return t;
}

static cudisc_status validate(const cudisc_coag_params *p, std::string &why)
{
    if (!p) { why = "params is NULL"; return CUDISC_EINVAL; }
    if (p->n_cells < 1) { why = "n_cells must be >= 1"; return CUDISC_EINVAL; }
    if (p->n_bins < 2) { why = "n_bins must be >= 2"; return CUDISC_EINVAL; }
    if (p->n_bins > cdc::kMaxBins) {
        why = "n_bins > 160 is not supported by this build";
        return CUDISC_ENOTSUP;
    }
    if (p->precision == CUDISC_MIXED_TF32 && p->n_bins > cdc::kMaxMixedBins) {
        why = "the mixed precision path supports n_bins <= 160";
        return CUDISC_ENOTSUP;
    }
    if (p->precision != CUDISC_FP64 && p->precision != CUDISC_MIXED_TF32) {
        why = "precision must be CUDISC_FP64 or CUDISC_MIXED_TF32";
        return CUDISC_EINVAL;
    }
    if (!p->mass_centres || !p->mass_edges) { why = "mass_centres / mass_edges are NULL"; return CUDISC_EINVAL; }
    if (!p->rho_gas || !p->T || !p->alpha || !p->R || !p->Z) {
        why = "rho_gas, T, alpha, R and Z must be device arrays";
        return CUDISC_EINVAL;
    }
    const int N = p->n_bins;
    for (int k = 0; k < N; k++) {
        double c = p->mass_centres[k];
        if (!(c > 0.0) || !std::isfinite(c)) { why = "mass_centres must be positive and finite"; return CUDISC_EINVAL; }
        if (k && !(c > p->mass_centres[k - 1])) { why = "mass_centres must be strictly increasing"; return CUDISC_EINVAL; }
        if (!(p->mass_edges[k] < c && c < p->mass_edges[k + 1])) {
            why = "mass_edges must bracket every centre: edge k < centre k < edge k+1";
            return CUDISC_EINVAL;
        }
    }
    if (!(p->mass_edges[0] > 0.0)) { why = "mass_edges[0] must be positive"; return CUDISC_EINVAL; }
    if (p->kernel_mode < 0 || p->kernel_mode > 2) { why = "kernel_mode out of range"; return CUDISC_EINVAL; }
    if (p->frag_mode < 0 || p->frag_mode > 2) { why = "frag_mode out of range"; return CUDISC_EINVAL; }
    if (p->split_mode < 0 || p->split_mode > 1) { why = "split_mode out of range"; return CUDISC_EINVAL; }
    if (!(p->rtol > 0.0) || !(p->atol_rel >= 0.0)) { why = "rtol must be > 0 and atol_rel >= 0"; return CUDISC_EINVAL; }
    if (p->max_substeps < 1) { why = "max_substeps must be >= 1"; return CUDISC_EINVAL; }
    if (p->mixed_pair < 0 || p->mixed_pair > 2) {
        why = "mixed_pair must be 0 (automatic), 1 (single CTAs) or 2 (CTA pairs)";
        return CUDISC_EINVAL;
    }
    if (p->mixed_cluster != 0 && p->mixed_cluster != 1 && p->mixed_cluster != 2 && p->mixed_cluster != 4 &&
        p->mixed_cluster != 8) {
        why = "mixed_cluster must be 0 (automatic), 1, 2, 4 or 8";
        return CUDISC_EINVAL;
    }
    if (p->max_sms < 0) { why = "max_sms must be >= 0 (0: all SMs)"; return CUDISC_EINVAL; }
    if (p->mixed_tile_stages < 0 || p->mixed_tile_stages > 8) {
        why = "mixed_tile_stages must be 0 (automatic) or 1..8";
        return CUDISC_EINVAL;
    }
    if (p->cost_order != 0 && p->cost_order != 1) {
        why = "cost_order must be 0 (previous step's cost order) or 1 (index order)";
        return CUDISC_EINVAL;
    }
    if (p->mixed_k_stages < 0 || p->mixed_k_stages > 4) {
        why = "mixed_k_stages must be 0 (automatic) or 1..4";
        return CUDISC_EINVAL;
    }
    if (p->vertical != 0 && p->vertical != 1) { why = "vertical must be 0 or 1"; return CUDISC_EINVAL; }
    if (!(p->rho_m > 0) || !(p->mu > 0) || !(p->Mstar > 0) || !(p->k_B > 0) || !(p->m_H > 0) ||
        !(p->G > 0) || !(p->sigma_H2 > 0)) {
        why = "rho_m, mu, Mstar, k_B, m_H, G and sigma_H2 must be positive";
        return CUDISC_EINVAL;
    }
    if (p->frag_mode == CUDISC_FRAG_PHYSICAL && !(p->v_frag > 0)) { why = "v_frag must be positive"; return CUDISC_EINVAL; }
    if (!(p->chi_im > 0)) { why = "chi_im must be positive"; return CUDISC_EINVAL; }
    return CUDISC_OK;
}

// Build every per-grid table on the host (FP64) and upload it.
static cudisc_status build_tables(cudisc_coag_ctx *c)
{
    const cudisc_coag_params &p = c->p;
    const int N = c->N;
    const std::vector<double> &m = c->h_m, &me = c->h_me;
    std::vector<double> minv(N), a(N);
    for (int k = 0; k < N; k++) {
        minv[k] = 1.0 / m[k];
        a[k] = std::cbrt(3.0 * m[k] / (4.0 * M_PI * p.rho_m));
    }
    // packed pairs p = i (i + 1) / 2 + j
    std::vector<unsigned int> pij(c->Np);
    for (int i = 0; i < N; i++)
        for (int j = 0; j <= i; j++) pij[i * (i + 1) / 2 + j] = ((unsigned)i << 16) | (unsigned)j;

    // fragment distribution table N_k(m^e_{l+1})
    std::vector<double> Ntab((size_t)N * N, 0.0);
    for (int l = 0; l < N; l++)
        for (int k = 0; k <= l; k++) Ntab[(size_t)l * N + k] = frag_share(me, p.eta_frag, k, l);

    // per-pair row of the redistribution, per unit n_i n_j K (1/2 at i = j):
    //   alpha_k: coagulation gain minus the loss of both grains,
    //   beta_k : remnant gain minus the coagulation gain (the part p_frag moves),
    //   Mf at l: fragment mass gathered per largest-fragment bin.
    // All coefficients are divided by m_i m_j so that they multiply rho_i rho_j K.
    std::vector<std::vector<std::pair<int, double2>>> rows(N);
    std::vector<std::vector<std::pair<int, double>>> frows(N);
    // mixed path dense tile image: per block b, hi then lo, NBP rows x 32 floats
    c->n_blk = 0;
    std::vector<int> blk_i, blk_j0;
    for (int i = 0; i < N; i++)
        for (int j0 = 0; j0 <= i; j0 += cdc::kBlkPairs) { blk_i.push_back(i); blk_j0.push_back(j0); }
    c->n_blk = (int)blk_i.size();
    const bool mixed = p.precision == CUDISC_MIXED_TF32;
    std::vector<float> tiles;
    const int NBP = cdc::mixed_nbp(N);
    if (mixed) tiles.assign((size_t)c->n_blk * 2 * NBP * cdc::kBlkElems, 0.0f);

    std::vector<dd> colA(N), colB(N);
    int blk = 0;
    for (int i = 0; i < N; i++) {
        for (int j = 0; j <= i; j++) {
            const int pp = i * (i + 1) / 2 + j;
            const double h = (i == j) ? 0.5 : 1.0;
            const double w = h / (m[i] * m[j]);
            const dd M = two_sum(m[i], m[j]);               // exact
            std::fill(colA.begin(), colA.end(), dd_of(0.0));
            std::fill(colB.begin(), colB.end(), dd_of(0.0));
            int kl, ku; dd fl, fu;
            two_bin_dd(m, M, p.split_mode, kl, ku, fl, fu);
            const dd cl = M * fl, cu = M * fu;
            colA[kl] = colA[kl] + cl; colA[ku] = colA[ku] + cu;
            colB[kl] = colB[kl] - cl; colB[ku] = colB[ku] - cu;
            colA[i] = colA[i] - dd_of(m[i]);
            colA[j] = colA[j] - dd_of(m[j]);
            const double mtar = m[i] >= m[j] ? m[i] : m[j];
            const double mim = m[i] >= m[j] ? m[j] : m[i];
            const dd cm = dd_of(p.chi_im) * dd_of(mim);
            const bool has_rem = dd_val(cm - dd_of(mtar)) < 0.0;
            const dd mrem = has_rem ? dd_of(mtar) - cm : dd_of(0.0);
            const double mx = has_rem ? dd_val(cm) : mtar;
            if (has_rem) {
                dd rl, ru;
                two_bin_dd(m, mrem, p.split_mode, kl, ku, rl, ru);
                colB[kl] = colB[kl] + mrem * rl;
                colB[ku] = colB[ku] + mrem * ru;
            }
            const double Mf = dd_val(M - mrem);
            // largest-fragment bin: smallest l with me[l+1] > mx
            int l = N - 1;
            if (me[N] > mx) {
                int lo = 0, hi = N - 1;
                while (lo < hi) {
                    int mid = (lo + hi) / 2;
                    if (me[mid + 1] > mx) hi = mid; else lo = mid + 1;
                }
                l = lo;
            }
            for (int k = 0; k < N; k++) {
                const double a_k = dd_val(colA[k]), b_k = dd_val(colB[k]);
                if (a_k != 0.0 || b_k != 0.0)
                    rows[k].push_back({pp, make_double2(a_k * w, b_k * w)});
            }
            frows[l].push_back({pp, Mf * w});
            if (mixed) {
                // dense columns of the contraction, against {K p_c, K p_f}:
                //   a: coagulation gain minus the loss of both grains,
                //   b: remnant and fragment gain (fragments folded in
                //      directly) minus the loss of both grains
                const int jb = j / cdc::kBlkPairs;
                const int b = blk + jb;
                const int t = j - jb * cdc::kBlkPairs;
                for (int k = 0; k < N; k++) {
                    double va = dd_val(colA[k]) * w;
                    dd vbd = colB[k] + colA[k];
                    if (k <= l) vbd = vbd + dd_of(Mf) * dd_of(Ntab[(size_t)l * N + k]);
                    double vb = dd_val(vbd) * w;
                    for (int s = 0; s < 2; s++) {
                        double v = s == 0 ? va : vb;
                        int e = 2 * t + s;                       // element in the row
                        float hi = bits_f(tf32_rn_bits((float)v));
                        float lo = bits_f(tf32_rn_bits((float)(v - (double)hi)));
                        int chunk = e >> 2;
                        size_t off = (size_t)k * 32 + (size_t)(((chunk ^ (k & 7)) << 2) | (e & 3));
                        size_t base = (size_t)b * 2 * NBP * 32;
                        tiles[base + off] = hi;
                        tiles[base + (size_t)NBP * 32 + off] = lo;
                    }
                }
            }
        }
        blk += (i + cdc::kBlkPairs) / cdc::kBlkPairs;
    }
    // CSR
    std::vector<int> row(N + 1, 0), ent_p, frow(N + 1, 0), fent_p;
    std::vector<double2> ent_ab;
    std::vector<double> fent_m;
    for (int k = 0; k < N; k++) {
        row[k] = (int)ent_p.size();
        for (auto &e : rows[k]) { ent_p.push_back(e.first); ent_ab.push_back(e.second); }
        frow[k] = (int)fent_p.size();
        for (auto &e : frows[k]) { fent_p.push_back(e.first); fent_m.push_back(e.second); }
    }
    row[N] = (int)ent_p.size();
    frow[N] = (int)fent_p.size();

    cudaStream_t s = c->stream;
    CUDA_TRY(c, upload(&c->d_m, m, s));
    CUDA_TRY(c, upload(&c->d_minv, minv, s));
    CUDA_TRY(c, upload(&c->d_a, a, s));
    CUDA_TRY(c, upload(&c->d_me, me, s));
    CUDA_TRY(c, upload(&c->d_pair_ij, pij, s));
    CUDA_TRY(c, upload(&c->d_row, row, s));
    CUDA_TRY(c, upload(&c->d_ent_p, ent_p, s));
    CUDA_TRY(c, upload(&c->d_ent_ab, ent_ab, s));
    CUDA_TRY(c, upload(&c->d_frow, frow, s));
    CUDA_TRY(c, upload(&c->d_fent_p, fent_p, s));
    CUDA_TRY(c, upload(&c->d_fent_m, fent_m, s));
    CUDA_TRY(c, upload(&c->d_Ntab, Ntab, s));
    CUDA_TRY(c, upload(&c->d_blk_i, blk_i, s));
    CUDA_TRY(c, upload(&c->d_blk_j0, blk_j0, s));
    if (mixed) {
        std::vector<float4> t4(tiles.size() / 4);
        std::memcpy(t4.data(), tiles.data(), tiles.size() * sizeof(float));
        CUDA_TRY(c, upload(&c->d_Btiles, t4, s));
    }
    return CUDISC_OK;
}

static void free_ctx(cudisc_coag_ctx *c)
{
    if (!c) return;
    void *ptrs[] = {c->d_m, c->d_minv, c->d_a, c->d_me, c->d_pair_ij, c->d_row, c->d_ent_p,
                    c->d_ent_ab, c->d_frow, c->d_fent_p, c->d_fent_m, c->d_Ntab, c->d_blk_i,
                    c->d_blk_j0, c->d_Btiles, c->d_prep, c->d_prep32, c->d_scal, c->d_K64,
                    c->d_K32, c->d_Kslot, c->d_out, c->d_work, c->d_counter, c->d_scal32, c->d_list,
                    c->d_spans, c->d_pending, c->d_host_state, c->d_order};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (cudaEvent_t &ev : c->evb)
        if (ev) cudaEventDestroy(ev);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_copied) cudaEventDestroy(c->ev_copied);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    cdc::vjp_free(c);
    delete c;
}

extern "C" {

const char *cudisc_coag_version(void) { return "cudisc-coag-b300 0.1 (sm_103a)"; }

const char *cudisc_coag_last_error(const cudisc_coag_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_thread_err.c_str();
}

cudisc_status cudisc_coag_init(const cudisc_coag_params *params, cudisc_coag_ctx **out)
{
    g_thread_err.clear();
    if (!out) return fail(nullptr, CUDISC_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    cudisc_status st = validate(params, why);
    if (st != CUDISC_OK) return fail(nullptr, st, why);
    cudisc_coag_ctx *c = new cudisc_coag_ctx();
    c->p = *params;
    c->stream = (cudaStream_t)params->stream;
    c->N = params->n_bins;
    c->Np = c->N * (c->N + 1) / 2;
    c->n_cells = params->n_cells;
    c->h_m.assign(params->mass_centres, params->mass_centres + c->N);
    c->h_me.assign(params->mass_edges, params->mass_edges + c->N + 1);
    // the stored pointers to host mass arrays are not kept
    c->p.mass_centres = nullptr;
    c->p.mass_edges = nullptr;
    st = build_tables(c);
    if (st != CUDISC_OK) { g_thread_err = c->err; free_ctx(c); return st; }
    const size_t nc = (size_t)c->n_cells, N = (size_t)c->N;
    cudaError_t e;
    e = cudaMalloc(&c->d_prep, nc * cdc::PF_COUNT * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_prep32, nc * cdc::P3_COUNT * N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scal, nc * sizeof(cdc::CellScal));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scal32, nc * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_out, nc * sizeof(CellOut));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_list, nc * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_order, nc * sizeof(int));
    if (e == cudaSuccess) {
        iota_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, c->stream>>>((int)nc, c->d_order);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMalloc(&c->d_spans, nc * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_pending, nc * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->d_pending, 0, nc * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->d_counter, 0, 64 * sizeof(int));
    if (e == cudaSuccess) {
        if (params->precision == CUDISC_FP64)
            e = cudaMalloc(&c->d_K64, nc * (size_t)c->Np * sizeof(double2));
        else
        {
            const bool fits = cdc::mixed_layout(c->n_cells, c->N, params->mixed_cluster, params->max_sms,
                                                params->mixed_pair, params->mixed_tile_stages,
                                                params->mixed_k_stages, &c->mix_P, &c->mix_G, &c->mix_C,
                                                &c->mix_pair);
            if (!fits && (params->mixed_tile_stages || params->mixed_k_stages)) {
                free_ctx(c);
                return fail(nullptr, CUDISC_EINVAL,
                            "mixed_tile_stages / mixed_k_stages do not fit the shared memory at this size");
            }
            // zeroed once: groups of four slots that lie wholly past a block's
            // diagonal are never written by the kernel builder
            const size_t k32 = (size_t)c->n_cells * c->n_blk * cdc::kBlkPairs * sizeof(float2);
            e = cudaMalloc(&c->d_K32, k32);
            if (e == cudaSuccess) e = cudaMemset(c->d_K32, 0, k32);
            // the slot groups' tables: [group][block][8 chunks][64 slots] x 16 B
            // (zeroed: slots that never hold a cell multiply zero stage inputs by it)
            const size_t kslot = (size_t)c->mix_G * c->n_blk * 8 * 64 * sizeof(float4);
            if (e == cudaSuccess) e = cudaMalloc(&c->d_Kslot, kslot);
            if (e == cudaSuccess) e = cudaMemset(c->d_Kslot, 0, kslot);
        }
    }
    if (e == cudaSuccess && params->precision == CUDISC_MIXED_TF32) {
        c->work_bytes = cdc::mixed_workspace_bytes(c->n_cells, c->N, c->mix_P, params->max_sms, c->mix_pair,
                                                   params->mixed_tile_stages, params->mixed_k_stages);
        e = cudaMalloc(&c->d_work, c->work_bytes);
    }
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    for (cudaEvent_t &ev : c->evb)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_stats, kStatsOff + (size_t)c->n_cells * sizeof(cdc::CellOut));
    if (e != cudaSuccess) {
        cuda_fail(c, e, "cudisc_coag_init: workspace allocation");
        st = (e == cudaErrorMemoryAllocation) ? CUDISC_ENOMEM : CUDISC_ECUDA;
        free_ctx(c);
        return st;
    }
    st = cudisc_coag_build_kernel(c);
    if (st != CUDISC_OK) { g_thread_err = c->err; free_ctx(c); return st; }
    *out = c;
    return CUDISC_OK;
}

void cudisc_coag_destroy(cudisc_coag_ctx *ctx) { free_ctx(ctx); }

cudisc_status cudisc_coag_get_timings(const cudisc_coag_ctx *c, cudisc_timings *out)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!out) return CUDISC_EINVAL;
    out->prep_ms = c->t_prep;
    out->kbuild_ms = c->t_kbuild;
    out->step_ms = c->t_step;
    out->vjp_ms = c->t_vjp;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_mixed_cluster(const cudisc_coag_ctx *c, int *cluster, int *groups)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!cluster || !groups) return CUDISC_EINVAL;
    const bool mixed = c->p.precision == CUDISC_MIXED_TF32;
    *cluster = mixed ? c->mix_P : 0;
    *groups = mixed ? c->mix_G : 0;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_mixed_pair(const cudisc_coag_ctx *c, int *pair)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!pair) return CUDISC_EINVAL;
    *pair = c->p.precision == CUDISC_MIXED_TF32 ? c->mix_pair : 0;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_mixed_rings(const cudisc_coag_ctx *c, int *tile_stages, int *k_stages, int *state_in_smem)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!tile_stages || !k_stages || !state_in_smem) return CUDISC_EINVAL;
    *tile_stages = *k_stages = *state_in_smem = 0;
    if (c->p.precision == CUDISC_MIXED_TF32)
        cdc::mixed_rings(c->n_cells, c->N, c->mix_P, c->p.max_sms, c->mix_pair, c->p.mixed_tile_stages,
                         c->p.mixed_k_stages, tile_stages, k_stages, state_in_smem);
    return CUDISC_OK;
}

cudisc_status cudisc_coag_build_kernel(cudisc_coag_ctx *c)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    CUDA_TRY(c, cudaEventRecord(c->evb[0], c->stream));
    CUDA_TRY(c, cdc::launch_prep(c));
    CUDA_TRY(c, cudaEventRecord(c->evb[1], c->stream));
    CUDA_TRY(c, cdc::launch_kbuild(c));
    CUDA_TRY(c, cudaEventRecord(c->evb[2], c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, c->evb[0], c->evb[1]);
    cudaEventElapsedTime(&b, c->evb[1], c->evb[2]);
    c->t_prep = a;
    c->t_kbuild = b;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_build_kernel_async(cudisc_coag_ctx *c)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    CUDA_TRY(c, cdc::launch_prep(c));
    CUDA_TRY(c, cdc::launch_kbuild(c));
    return CUDISC_OK;
}

cudisc_status cudisc_coag_set_adjoint_precision(cudisc_coag_ctx *c, int precision)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (precision != CUDISC_ADJOINT_FP64 && precision != CUDISC_ADJOINT_DOUBLE_FLOAT)
        return fail(c, CUDISC_EINVAL, "adjoint precision must be CUDISC_ADJOINT_FP64 or CUDISC_ADJOINT_DOUBLE_FLOAT");
    c->adj_prec = precision;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_set_v_frag(cudisc_coag_ctx *c, double v_frag)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!(v_frag > 0.0) || !std::isfinite(v_frag))
        return fail(c, CUDISC_EINVAL, "v_frag must be positive and finite");
    c->p.v_frag = v_frag;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_get_kernel(cudisc_coag_ctx *c, double *K_out, double *KF_out)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!K_out || !KF_out) return fail(c, CUDISC_EINVAL, "K_out / KF_out are NULL");
    CUDA_TRY(c, cdc::launch_get_kernel(c, K_out, KF_out));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CUDISC_OK;
}

cudisc_status cudisc_coag_rhs(cudisc_coag_ctx *c, const double *rho, double *drho)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!rho || !drho) return fail(c, CUDISC_EINVAL, "rho / drho_dt are NULL");
    if (c->p.precision == CUDISC_FP64) CUDA_TRY(c, cdc::launch_rhs_fp64(c, rho, drho));
    else CUDA_TRY(c, cdc::launch_rhs_mixed(c, rho, drho));
    return CUDISC_OK;
}

cudisc_status cudisc_coag_set_records(cudisc_coag_ctx *c, double *dt_log, long long log_cap,
                                      long long *n_log, int *status)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (dt_log && log_cap < 1) return fail(c, CUDISC_EINVAL, "log_cap must be >= 1 with dt_log");
    c->rec_dt = dt_log;
    c->rec_cap = dt_log ? log_cap : 0;
    c->rec_n = n_log;
    c->rec_status = status;
    return CUDISC_OK;
}

static cudisc_status finish_step(cudisc_coag_ctx *c, cudisc_step_stats *stats)
{
    // the status word and the per-cell results, read into pinned memory
    // behind the integration, then one synchronisation
    int *h_err = (int *)c->h_stats;
    const CellOut *h = (const CellOut *)((char *)c->h_stats + kStatsOff);
    CUDA_TRY(c, cudaMemcpyAsync(h_err, c->d_counter + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync((void *)h, c->d_out, (size_t)c->n_cells * sizeof(CellOut), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int dev_err = *h_err;
    if (dev_err != 0) {
        char buf[128];
        std::snprintf(buf, sizeof(buf), "a bounded device wait ran out (code %d); results are invalid", dev_err);
        return fail(c, CUDISC_ECUDA, buf);
    }
    cudisc_step_stats s;
    std::memset(&s, 0, sizeof(s));
    for (int i = 0; i < c->n_cells; i++) {
        const CellOut &o = h[i];
        s.accepted += o.n_acc;
        s.rejected += o.n_rej;
        if (o.n_acc > s.max_accepted) s.max_accepted = o.n_acc;
        if (o.status != 0) s.n_failed++;
        if (o.status > s.worst_status) s.worst_status = o.status;
        if (o.mass_err > s.mass_err_max) s.mass_err_max = o.mass_err;
    }
    float ms = 0.f;
    if (c->timed) cudaEventElapsedTime(&ms, c->ev0, c->ev1);   // untimed (asynchronous) steps report 0
    s.elapsed_ms = ms;
    c->t_step = ms;
    if (stats) *stats = s;
    if (s.worst_status != 0) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "%d of %d cells failed; worst per-cell status %d",
                      s.n_failed, c->n_cells, s.worst_status);
        c->err = buf;
        return (cudisc_status)s.worst_status;
    }
    return CUDISC_OK;
}

// Issue one integration on the context's stream (no synchronisation).
static cudisc_status issue_step(cudisc_coag_ctx *c, double *rho, double t_span, double *dt_cell, bool timed)
{
    if (!rho) return fail(c, CUDISC_EINVAL, "rho is NULL");
    if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(c, CUDISC_EINVAL, "t_span must be positive and finite");
    if (timed) CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    cdc::WorkList wl;                 // every cell, in the previous step's cost order
    if (c->p.cost_order == 0) wl.cells = c->d_order;
    if (c->p.precision == CUDISC_FP64)
        CUDA_TRY(c, cdc::launch_step_fp64(c, rho, t_span, dt_cell, nullptr, nullptr, 0, wl));
    else
        CUDA_TRY(c, cdc::launch_step_mixed(c, rho, t_span, dt_cell, nullptr, nullptr, 0, wl));
    if (timed) CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    if (c->p.cost_order == 0) {
        cost_order_kernel<<<1, 1024, 0, c->stream>>>(c->n_cells, c->d_out, c->d_order);
        CUDA_TRY(c, cudaGetLastError());
    }
    c->timed = timed;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_step(cudisc_coag_ctx *c, double *rho, double t_span, double *dt_cell,
                               cudisc_step_stats *stats)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    cudisc_status st = issue_step(c, rho, t_span, dt_cell, true);
    if (st != CUDISC_OK) return st;
    return finish_step(c, stats);
}

cudisc_status cudisc_coag_step_host(cudisc_coag_ctx *c, const double *rho_in, double *rho_out, double t_span,
                                    int rebuild, cudisc_step_stats *stats)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!rho_in || !rho_out) return fail(c, CUDISC_EINVAL, "rho_in and rho_out must be host arrays");
    if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(c, CUDISC_EINVAL, "t_span must be positive and finite");
    const size_t bytes = (size_t)c->n_cells * c->N * sizeof(double);
    if (!c->d_host_state) {
        CUDA_TRY(c, cudaMalloc(&c->d_host_state, bytes));
        CUDA_TRY(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
    }
    if (rebuild) {
        // the kernel tables depend on the gas arrays only: the state's copy
        // runs on a second stream beside their build, forked after the
        // stream's earlier work and joined before the integration
        CUDA_TRY(c, cudaEventRecord(c->ev_fork, c->stream));
        CUDA_TRY(c, cudaStreamWaitEvent(c->copy_stream, c->ev_fork, 0));
        CUDA_TRY(c, cudaMemcpyAsync(c->d_host_state, rho_in, bytes, cudaMemcpyHostToDevice, c->copy_stream));
        CUDA_TRY(c, cudaEventRecord(c->ev_copied, c->copy_stream));
        const cudisc_status sb = cudisc_coag_build_kernel_async(c);
        CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_copied, 0));
        if (sb != CUDISC_OK) return sb;
    } else {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_host_state, rho_in, bytes, cudaMemcpyHostToDevice, c->stream));
    }
    cudisc_status st = issue_step(c, c->d_host_state, t_span, nullptr, true);
    if (st != CUDISC_OK) return st;
    CUDA_TRY(c, cudaMemcpyAsync(rho_out, c->d_host_state, bytes, cudaMemcpyDeviceToHost, c->stream));
    return finish_step(c, stats);
}

// Build the work list on the device, then one timed integration over it.
static cudisc_status issue_worklist_step(cudisc_coag_ctx *c, double *rho, const double *span_in,
                                         double dt_global, double trigger, double *dt_cell)
{
    if (!rho) return fail(c, CUDISC_EINVAL, "rho is NULL");
    CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->d_counter + 3, 0, sizeof(int), c->stream));
    worklist_kernel<<<(c->n_cells + 255) / 256, 256, 0, c->stream>>>(
        c->n_cells, span_in, c->d_pending, dt_global, trigger, dt_cell, c->d_spans, c->d_list, c->d_counter + 3,
        c->d_out, c->rec_n, c->rec_status);
    CUDA_TRY(c, cudaGetLastError());
    cdc::WorkList wl;
    wl.cells = c->d_list;
    wl.count = c->d_counter + 3;
    wl.spans = c->d_spans;
    if (c->p.precision == CUDISC_FP64)
        CUDA_TRY(c, cdc::launch_step_fp64(c, rho, 1.0, dt_cell, nullptr, nullptr, 0, wl));
    else
        CUDA_TRY(c, cdc::launch_step_mixed(c, rho, 1.0, dt_cell, nullptr, nullptr, 0, wl));
    CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    c->timed = true;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_step_spans(cudisc_coag_ctx *c, double *rho, const double *t_span, double *dt_cell,
                                     cudisc_step_stats *stats)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!t_span) return fail(c, CUDISC_EINVAL, "t_span is NULL");
    cudisc_status st = issue_worklist_step(c, rho, t_span, 0.0, 1.0, dt_cell);
    if (st != CUDISC_OK) return st;
    return finish_step(c, stats);
}

cudisc_status cudisc_coag_subcycle(cudisc_coag_ctx *c, double *rho, double dt_global, double trigger,
                                   double *dt_cell, cudisc_step_stats *stats)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!(dt_global >= 0.0) || !std::isfinite(dt_global))
        return fail(c, CUDISC_EINVAL, "dt_global must be >= 0 and finite");
    if (!(trigger > 0.0) || !std::isfinite(trigger)) return fail(c, CUDISC_EINVAL, "trigger must be positive and finite");
    cudisc_status st = issue_worklist_step(c, rho, nullptr, dt_global, trigger, dt_cell);
    if (st != CUDISC_OK) return st;
    return finish_step(c, stats);
}

cudisc_status cudisc_coag_subcycle_pending(cudisc_coag_ctx *c, double *pending, int reset)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    const size_t bytes = (size_t)c->n_cells * sizeof(double);
    if (pending) CUDA_TRY(c, cudaMemcpyAsync(pending, c->d_pending, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (reset) CUDA_TRY(c, cudaMemsetAsync(c->d_pending, 0, bytes, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CUDISC_OK;
}

cudisc_status cudisc_hse_rho_gas(int n_R, int n_Z, const double *R, const double *Z, const double *T,
                                 const double *V, const double *R_edges, const double *Sigma_g, double mu,
                                 double m_H, double k_B, double GM, double *rho_gas, void *stream)
{
    g_thread_err.clear();
    if (n_R < 1 || n_Z < 1) return fail(nullptr, CUDISC_EINVAL, "n_R and n_Z must be >= 1");
    if ((long long)n_R * n_Z > (1ll << 40)) return fail(nullptr, CUDISC_EINVAL, "n_R x n_Z is too large");
    if (!R || !Z || !T || !V || !R_edges || !Sigma_g || !rho_gas)
        return fail(nullptr, CUDISC_EINVAL, "R, Z, T, V, R_edges, Sigma_g and rho_gas must be device arrays");
    const double pos[4] = {mu, m_H, k_B, GM};
    for (double v : pos)
        if (!(v > 0.0) || !std::isfinite(v)) return fail(nullptr, CUDISC_EINVAL, "mu, m_H, k_B and GM must be positive");
    cudaError_t e = cdc::launch_hse(n_R, n_Z, R, Z, T, V, R_edges, Sigma_g, mu, m_H, k_B, GM, rho_gas,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudisc_hse_rho_gas");
    return CUDISC_OK;
}

cudisc_status cudisc_dust_source_update(int n_species, int n_cells, double *Q, const double *P_n, double h,
                                        const double *R, const double *Z, const double *rho_g,
                                        const double *c_s, const double *v_g, const double *a, double rho_m,
                                        double GM, void *stream)
{
    g_thread_err.clear();
    if (n_species < 1 || n_cells < 1) return fail(nullptr, CUDISC_EINVAL, "n_species and n_cells must be >= 1");
    if (!Q || !P_n || !R || !Z || !rho_g || !c_s || !v_g || !a)
        return fail(nullptr, CUDISC_EINVAL, "Q, P_n, R, Z, rho_g, c_s, v_g and a must be device arrays");
    if (!(h >= 0.0) || !std::isfinite(h)) return fail(nullptr, CUDISC_EINVAL, "h must be >= 0 and finite");
    if (!(rho_m > 0.0) || !(GM >= 0.0) || !std::isfinite(rho_m) || !std::isfinite(GM))
        return fail(nullptr, CUDISC_EINVAL, "rho_m must be positive and GM >= 0");
    cudaError_t e = cdc::launch_dust_source(n_species, n_cells, Q, P_n, h, R, Z, rho_g, c_s, v_g, a, rho_m, GM,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudisc_dust_source_update");
    return CUDISC_OK;
}

cudisc_status cudisc_dust_cfl_dt(int n_species, int n_cells, const double *P, const double *dR, const double *dZ,
                                 const double *nu, const double *Sc, double C_adv, double C_diff, double *dt_out,
                                 void *stream)
{
    g_thread_err.clear();
    if (n_species < 1 || n_cells < 1) return fail(nullptr, CUDISC_EINVAL, "n_species and n_cells must be >= 1");
    if (!P || !dR || !dZ || !nu || !Sc || !dt_out)
        return fail(nullptr, CUDISC_EINVAL, "P, dR, dZ, nu, Sc and dt_out must be device arrays");
    if (!(C_adv > 0.0) || !(C_diff > 0.0) || !std::isfinite(C_adv) || !std::isfinite(C_diff))
        return fail(nullptr, CUDISC_EINVAL, "C_adv and C_diff must be positive");
    cudaError_t e = cdc::launch_dust_cfl(n_species, n_cells, P, dR, dZ, nu, Sc, C_adv, C_diff, dt_out,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudisc_dust_cfl_dt");
    return CUDISC_OK;
}

cudisc_status cudisc_coag_step_async(cudisc_coag_ctx *c, double *rho, double t_span, double *dt_cell)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    return issue_step(c, rho, t_span, dt_cell, false);
}

cudisc_status cudisc_coag_step_wait(cudisc_coag_ctx *c, cudisc_step_stats *stats)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    return finish_step(c, stats);
}

cudisc_status cudisc_coag_step_static_scratch(cudisc_coag_ctx *c, double *rho, double t_span,
                                              double *dt_cell, cudisc_step_stats *stats)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!rho) return fail(c, CUDISC_EINVAL, "rho is NULL");
    if (c->p.precision != CUDISC_MIXED_TF32)
        return fail(c, CUDISC_EINVAL, "cudisc_coag_step_static_scratch needs a CUDISC_MIXED_TF32 context");
    if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(c, CUDISC_EINVAL, "t_span must be positive and finite");
    bool too_big = false;
    CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    CUDA_TRY(c, cdc::launch_step_mixed_static(c, rho, t_span, dt_cell, &too_big));
    if (too_big) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "problem needs more integrator scratch than the fixed %zu MiB static array; "
                      "use cudisc_coag_step", cdc::static_scratch_bytes() >> 20);
        return fail(c, CUDISC_ENOTSUP, buf);
    }
    CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    c->timed = true;
    return finish_step(c, stats);
}

cudisc_status cudisc_coag_set_fault_injection(cudisc_coag_ctx *c, long long wait_cycles, int withhold)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (wait_cycles < 0 || (withhold != 0 && withhold != 1))
        return fail(c, CUDISC_EINVAL, "wait_cycles must be >= 0 and withhold 0 or 1");
    if (withhold && wait_cycles == 0)
        return fail(c, CUDISC_EINVAL, "withhold needs a short wait_cycles (the default limit is ~2 s)");
    c->inject_wait_cycles = wait_cycles;
    c->inject_withhold = withhold;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_scratch_bytes(const cudisc_coag_ctx *c, size_t *bytes)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!bytes) return CUDISC_EINVAL;
    *bytes = c->p.precision == CUDISC_MIXED_TF32
                 ? cdc::mixed_scratch_bytes(c->n_cells, c->N, c->mix_P, c->p.max_sms, c->mix_pair,
                                            c->p.mixed_tile_stages, c->p.mixed_k_stages)
                 : 0;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_replay(cudisc_coag_ctx *c, double *rho, const double *hs,
                                 const long long *n_h, long long stride)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!rho || !hs || !n_h) return fail(c, CUDISC_EINVAL, "rho, hs and n_h must be device arrays");
    if (stride < 1) return fail(c, CUDISC_EINVAL, "stride must be >= 1");
    CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    if (c->p.precision == CUDISC_FP64)
        CUDA_TRY(c, cdc::launch_step_fp64(c, rho, 1.0, nullptr, hs, n_h, stride));
    else
        CUDA_TRY(c, cdc::launch_step_mixed(c, rho, 1.0, nullptr, hs, n_h, stride));
    CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    c->timed = true;
    return finish_step(c, nullptr);
}

cudisc_status cudisc_coag_vjp(cudisc_coag_ctx *c, const double *rho0, double t_span,
                              const double *hs, const long long *n_h, long long stride,
                              const double *grad_rhoT, double *grad_rho0, double *grad_alpha,
                              double *grad_vfrag)
{
    if (!c) return fail(nullptr, CUDISC_EINVAL, "ctx is NULL");
    if (!rho0 || !grad_rhoT || !grad_rho0)
        return fail(c, CUDISC_EINVAL, "rho0, grad_rhoT and grad_rho0 must be device arrays");
    if (!cdc::vjp_fits(c))
        return fail(c, CUDISC_ENOTSUP, "n_bins too large for the adjoint's per-cell shared memory");
    const size_t nc = (size_t)c->n_cells;
    const double *H = hs;
    const long long *NH = n_h;
    long long str = stride;
    std::vector<long long> hn(nc);
    if (!hs) {
        // the step sequence of a fresh adaptive integration from rho0
        if (!(t_span > 0.0) || !std::isfinite(t_span))
            return fail(c, CUDISC_EINVAL, "t_span must be positive and finite");
        long long cap = std::max<long long>(1, std::min<long long>(c->p.max_substeps, 4096));
        for (int attempt = 0; attempt < 2; attempt++) {
            double *dt = nullptr, *tmp = nullptr;
            long long *nn = nullptr;
            int *sts = nullptr;
            CUDA_TRY(c, cdc::vjp_records(c, cap, &dt, &nn, &sts, &tmp));
            CUDA_TRY(c, cudaMemcpyAsync(tmp, rho0, nc * c->N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->stream));
            double *u_dt = c->rec_dt;
            long long u_cap = c->rec_cap, *u_n = c->rec_n;
            int *u_st = c->rec_status;
            c->rec_dt = dt; c->rec_cap = cap; c->rec_n = nn; c->rec_status = sts;
            cudaError_t e = cudaEventRecord(c->ev0, c->stream);
            if (e == cudaSuccess)
                e = c->p.precision == CUDISC_FP64
                        ? cdc::launch_step_fp64(c, tmp, t_span, nullptr, nullptr, nullptr, 0)
                        : cdc::launch_step_mixed(c, tmp, t_span, nullptr, nullptr, nullptr, 0);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev1, c->stream);
            c->rec_dt = u_dt; c->rec_cap = u_cap; c->rec_n = u_n; c->rec_status = u_st;
            if (e != cudaSuccess) return cuda_fail(c, e, "cudisc_coag_vjp: forward integration");
            cudisc_status st = finish_step(c, nullptr);
            if (st != CUDISC_OK) return st;
            CUDA_TRY(c, cudaMemcpy(hn.data(), nn, nc * sizeof(long long), cudaMemcpyDeviceToHost));
            const long long mx = *std::max_element(hn.begin(), hn.end());
            H = dt; NH = nn; str = cap;
            if (mx <= cap) break;
            cap = mx;
        }
    } else {
        if (!n_h) return fail(c, CUDISC_EINVAL, "n_h must be a device array with hs");
        if (stride < 1) return fail(c, CUDISC_EINVAL, "stride must be >= 1");
    }
    CUDA_TRY(c, cudaMemcpy(hn.data(), NH, nc * sizeof(long long), cudaMemcpyDeviceToHost));
    long long mx = 0;
    for (long long v : hn) {
        if (v < 0 || v > str) return fail(c, CUDISC_EINVAL, "n_h entries must lie in [0, stride]");
        mx = std::max(mx, v);
    }
    CUDA_TRY(c, cdc::vjp_prepare(c, mx));
    CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    CUDA_TRY(c, cdc::launch_vjp(c, rho0, H, NH, str, grad_rhoT, grad_rho0, grad_alpha, grad_vfrag));
    CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->t_vjp = ms;
    int worst = 0;
    CUDA_TRY(c, cdc::vjp_worst_status(c, &worst));
    if (worst != 0) return fail(c, (cudisc_status)worst, "non-finite adjoint in some cell");
    return CUDISC_OK;
}

// ---- batched discs -------------------------------------------------------

} // extern "C"

struct cudisc_coag_batch {
    std::vector<cudisc_coag_ctx *> ctx;
    std::vector<cudaStream_t> stream;
    std::vector<cudaEvent_t> done;
    cudaEvent_t ready = nullptr;
};

static void free_batch(cudisc_coag_batch *b)
{
    if (!b) return;
    for (cudisc_coag_ctx *c : b->ctx) free_ctx(c);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : b->stream)
        if (s) cudaStreamDestroy(s);
    if (b->ready) cudaEventDestroy(b->ready);
    delete b;
}

extern "C" {

cudisc_status cudisc_coag_init_batched(const cudisc_coag_params *params, int n_discs, cudisc_coag_batch **out)
{
    g_thread_err.clear();
    if (!out) return fail(nullptr, CUDISC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || n_discs < 1) return fail(nullptr, CUDISC_EINVAL, "params must hold n_discs >= 1 discs");
    for (int i = 0; i < n_discs; i++) {
        std::string why;
        const cudisc_status st = validate(&params[i], why);
        if (st != CUDISC_OK) return fail(nullptr, st, "disc " + std::to_string(i) + ": " + why);
    }
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // SM shares in proportion to n_cells x n_bins^2 (the work of a pass), at
    // least one each, handed out largest remainder first
    std::vector<double> w(n_discs);
    double W = 0.0;
    for (int i = 0; i < n_discs; i++) {
        w[i] = (double)params[i].n_cells * params[i].n_bins * params[i].n_bins;
        W += w[i];
    }
    std::vector<int> sms(n_discs, 1);
    int left = n_sm - n_discs;
    if (left > 0) {
        std::vector<std::pair<double, int>> rem;
        int given = 0;
        for (int i = 0; i < n_discs; i++) {
            const double q = left * w[i] / W;
            const int f = (int)q;
            sms[i] += f;
            given += f;
            rem.push_back({q - f, i});
        }
        std::sort(rem.begin(), rem.end(), [](const std::pair<double, int> &x, const std::pair<double, int> &y) {
            return x.first > y.first;
        });
        for (int k = 0; k < left - given && k < n_discs; k++) sms[rem[k].second]++;
    }
    cudisc_coag_batch *b = new cudisc_coag_batch();
    cudaError_t e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
    for (int i = 0; i < n_discs && e == cudaSuccess; i++) {
        cudaStream_t s = nullptr;
        cudaEvent_t d = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
        b->stream.push_back(s);
        b->done.push_back(d);
    }
    if (e != cudaSuccess) {
        free_batch(b);
        return fail(nullptr, CUDISC_ECUDA, std::string("cudisc_coag_init_batched: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < n_discs; i++) {
        cudisc_coag_params p = params[i];
        p.stream = b->stream[i];
        p.max_sms = sms[i];
        cudisc_coag_ctx *c = nullptr;
        const cudisc_status st = cudisc_coag_init(&p, &c);
        if (st != CUDISC_OK) {
            const std::string msg = "disc " + std::to_string(i) + ": " + g_thread_err;
            free_batch(b);
            return fail(nullptr, st, msg);
        }
        b->ctx.push_back(c);
    }
    *out = b;
    return CUDISC_OK;
}

cudisc_status cudisc_coag_batch_ctx(cudisc_coag_batch *b, int i, cudisc_coag_ctx **ctx)
{
    if (!b || !ctx) return fail(nullptr, CUDISC_EINVAL, "batch or ctx is NULL");
    if (i < 0 || i >= (int)b->ctx.size()) return fail(nullptr, CUDISC_EINVAL, "disc index out of range");
    *ctx = b->ctx[i];
    return CUDISC_OK;
}

cudisc_status cudisc_coag_batch_build_kernel(cudisc_coag_batch *b)
{
    if (!b) return fail(nullptr, CUDISC_EINVAL, "batch is NULL");
    // each build synchronises its own stream only; issue them all, then wait
    cudisc_status worst = CUDISC_OK;
    for (cudisc_coag_ctx *c : b->ctx) {
        const cudisc_status st = cudisc_coag_build_kernel(c);
        if (st != CUDISC_OK && worst == CUDISC_OK) worst = st;
    }
    return worst;
}

cudisc_status cudisc_coag_batch_step(cudisc_coag_batch *b, double *const *rho, double t_span,
                                     double *const *dt_cell, void *stream, cudisc_step_stats *stats)
{
    if (!b) return fail(nullptr, CUDISC_EINVAL, "batch is NULL");
    if (!rho) return fail(nullptr, CUDISC_EINVAL, "rho is NULL");
    const int n = (int)b->ctx.size();
    cudaStream_t s0 = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(b->ready, s0);
    if (e != cudaSuccess) return fail(nullptr, CUDISC_ECUDA, cudaGetErrorString(e));
    // issue every disc on its own stream, after the caller's queued work
    cudisc_status worst = CUDISC_OK;
    std::vector<bool> issued(n, false);
    for (int i = 0; i < n; i++) {
        cudisc_coag_ctx *c = b->ctx[i];
        e = cudaStreamWaitEvent(b->stream[i], b->ready, 0);
        if (e != cudaSuccess) { cuda_fail(c, e, "batch step"); worst = CUDISC_ECUDA; continue; }
        const cudisc_status st = issue_step(c, rho[i], t_span, dt_cell ? dt_cell[i] : nullptr, true);
        if (st != CUDISC_OK) { if (worst == CUDISC_OK || st > worst) worst = st; continue; }
        issued[i] = true;
        e = cudaEventRecord(b->done[i], b->stream[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, b->done[i], 0);
        if (e != cudaSuccess) { cuda_fail(c, e, "batch step"); worst = CUDISC_ECUDA; }
    }
    // then collect each disc (its stream is already running)
    for (int i = 0; i < n; i++) {
        if (!issued[i]) {
            if (stats) std::memset(&stats[i], 0, sizeof(cudisc_step_stats));
            continue;
        }
        const cudisc_status st = finish_step(b->ctx[i], stats ? &stats[i] : nullptr);
        if (st != CUDISC_OK && (worst == CUDISC_OK || st > worst)) worst = st;
    }
    return worst;
}

cudisc_status cudisc_coag_batch_step_async(cudisc_coag_batch *b, double *const *rho, double t_span,
                                           double *const *dt_cell, void *stream)
{
    if (!b) return fail(nullptr, CUDISC_EINVAL, "batch is NULL");
    if (!rho) return fail(nullptr, CUDISC_EINVAL, "rho is NULL");
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; i++)
        if (!rho[i]) return fail(nullptr, CUDISC_EINVAL, "rho[" + std::to_string(i) + "] is NULL");
    if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(nullptr, CUDISC_EINVAL, "t_span must be positive and finite");
    cudaStream_t s0 = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(b->ready, s0);
    if (e != cudaSuccess) return fail(nullptr, CUDISC_ECUDA, cudaGetErrorString(e));
    // fork every disc's stream from s0 and join it back: the whole batch is
    // one span of s0's work (and one graph when s0 is being captured)
    for (int i = 0; i < n; i++) {
        cudisc_coag_ctx *c = b->ctx[i];
        CUDA_TRY(c, cudaStreamWaitEvent(b->stream[i], b->ready, 0));
        const cudisc_status st = issue_step(c, rho[i], t_span, dt_cell ? dt_cell[i] : nullptr, false);
        if (st != CUDISC_OK) return st;
        CUDA_TRY(c, cudaEventRecord(b->done[i], b->stream[i]));
        CUDA_TRY(c, cudaStreamWaitEvent(s0, b->done[i], 0));
    }
    return CUDISC_OK;
}

cudisc_status cudisc_coag_batch_step_wait(cudisc_coag_batch *b, cudisc_step_stats *stats)
{
    if (!b) return fail(nullptr, CUDISC_EINVAL, "batch is NULL");
    cudisc_status worst = CUDISC_OK;
    for (size_t i = 0; i < b->ctx.size(); i++) {
        const cudisc_status st = finish_step(b->ctx[i], stats ? &stats[i] : nullptr);
        if (st != CUDISC_OK && (worst == CUDISC_OK || st > worst)) worst = st;
    }
    return worst;
}

void cudisc_coag_batch_destroy(cudisc_coag_batch *b) { free_batch(b); }

// ---- shards for several GPUs ---------------------------------------------
//
// Cells (and whole discs) are independent during a coagulation call, so a
// job spreads over GPUs by giving each a contiguous range of them.  The
// ranges minimise the largest range cost: the smallest bottleneck B for
// which a greedy left-to-right fill (a new range once the next item would
// take the running sum past B) needs at most n_parts ranges is found by
// bisection between max(largest item, total / n_parts) and the total, and
// that fill gives the bounds.  Unused trailing ranges are empty.

static int greedy_parts(int n, const double *cost, double B, int *bounds, int n_parts)
{
    int parts = 1;
    double acc = 0.0;
    if (bounds) bounds[0] = 0;
    for (int i = 0; i < n; i++) {
        const double c = cost ? cost[i] : 1.0;
        if (acc > 0.0 && acc + c > B) {
            if (bounds && parts < n_parts) bounds[parts] = i;
            parts++;
            acc = c;
        } else {
            acc += c;
        }
    }
    if (bounds)
        for (int k = std::min(parts, n_parts); k <= n_parts; k++) bounds[k] = n;
    return parts;
}

cudisc_status cudisc_partition(int n_items, const double *cost, int n_parts, int *bounds)
{
    g_thread_err.clear();
    if (n_items < 0 || n_parts < 1) return fail(nullptr, CUDISC_EINVAL, "n_items must be >= 0 and n_parts >= 1");
    if (!bounds) return fail(nullptr, CUDISC_EINVAL, "bounds is NULL");
    double total = 0.0, big = 0.0;
    for (int i = 0; i < n_items; i++) {
        const double c = cost ? cost[i] : 1.0;
        if (!(c >= 0.0) || !std::isfinite(c)) return fail(nullptr, CUDISC_EINVAL, "costs must be finite and >= 0");
        total += c;
        big = std::max(big, c);
    }
    double lo = std::max(big, total / n_parts), hi = std::max(total, lo);
    if (greedy_parts(n_items, cost, lo, nullptr, n_parts) <= n_parts) hi = lo;
    for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; it++) {
        const double mid = 0.5 * (lo + hi);
        if (greedy_parts(n_items, cost, mid, nullptr, n_parts) <= n_parts) hi = mid;
        else lo = mid;
    }
    greedy_parts(n_items, cost, hi, bounds, n_parts);
    return CUDISC_OK;
}

} // extern "C"
