// FP64 path: Eq. (smol) evaluated as a gather over the sparse redistribution
// (every output bin k sums its coagulation, remnant and loss entries, then
// the fragment mass gathered per largest-fragment bin l is spread by
// N_k(m^e_{l+1}), the two-stage form of Sec. 5), and the Bogacki-Shampine
// 3(2) integrator with per-cell step control (Sec. 5, last paragraph).
//
// One CTA integrates one cell at a time, taking cells from a global work
// queue; the pair weights of the cell live in shared memory.
#include <algorithm>
#include <cmath>

#include "coag_internal.h"

namespace cdc {
namespace {

constexpr int kThreads = 256;
constexpr double A21 = 0.5, A32 = 0.75;
constexpr double B1 = 2.0 / 9.0, B2 = 1.0 / 3.0, B3 = 4.0 / 9.0;
constexpr double E1 = -5.0 / 72.0, E2 = 1.0 / 12.0, E3 = 1.0 / 9.0, E4 = -1.0 / 8.0;

struct StepArgs {
    DevTables t;
    const double2 *K64;
    double *rho;
    double t_span;
    double *dt_cell;
    double rtol, atol_rel;
    long long max_steps;
    const double *replay_h;
    const long long *replay_n;
    long long replay_stride;
    CellOut *out;
    int *counter;
    double *rec_dt;
    long long rec_cap;
    long long *rec_n;
    int *rec_status;
    WorkList wl;                // the cells to integrate and their spans
};

size_t smem_doubles(int N, int Np) { return 2 * (size_t)Np + 8 * (size_t)N + 32; }

// d rho / dt of one cell: x = state (smem), f = result (smem).
__device__ void rhs64(const DevTables &t, const double2 *__restrict__ Kc, const double *x,
                      double *f, double *Wa, double *Wb, double *fl)
{
    const int N = t.N, Np = t.Np;
    for (int p = threadIdx.x; p < Np; p += blockDim.x) {
        const unsigned int ij = __ldg(t.pair_ij + p);
        const double xx = x[ij >> 16] * x[ij & 0xffff];
        const double2 k = __ldg(Kc + p);
        Wa[p] = xx * k.x;          // rho_i rho_j K_ij
        Wb[p] = xx * k.y;          // rho_i rho_j K_ij p_frag,ij
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double acc = 0.0;
        const int e1 = __ldg(t.row + k + 1);
        for (int e = __ldg(t.row + k); e < e1; e++) {
            const int p = __ldg(t.ent_p + e);
            const double2 ab = __ldg(t.ent_ab + e);
            acc = fma(Wa[p], ab.x, acc);
            acc = fma(Wb[p], ab.y, acc);
        }
        double g = 0.0;
        const int q1 = __ldg(t.frow + k + 1);
        for (int e = __ldg(t.frow + k); e < q1; e++) g = fma(Wb[__ldg(t.fent_p + e)], __ldg(t.fent_m + e), g);
        f[k] = acc;
        fl[k] = g;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double acc = f[k];
        for (int l = k; l < N; l++) acc = fma(fl[l], __ldg(t.Ntab + (size_t)l * N + k), acc);
        f[k] = acc;
    }
    __syncthreads();
}

template <class Op>
__device__ double block_reduce(double v, double *red, Op op)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); i++) r = op(r, red[i]);
    return r;
}

struct MaxOp { __device__ double operator()(double a, double b) const { return a > b ? a : b; } };
struct MinOp { __device__ double operator()(double a, double b) const { return a < b ? a : b; } };

__global__ void __launch_bounds__(kThreads) rhs64_kernel(int c0, DevTables t,
                                                         const double2 *__restrict__ K64,
                                                         const double *__restrict__ rho,
                                                         double *__restrict__ drho)
{
    extern __shared__ double sm[];
    const int N = t.N, Np = t.Np;
    double *Wa = sm, *Wb = Wa + Np, *x = Wb + Np, *f = x + N, *fl = f + N;
    const int c = c0 + blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x) x[k] = rho[(size_t)c * N + k];
    __syncthreads();
    rhs64(t, K64 + (size_t)c * Np, x, f, Wa, Wb, fl);
    for (int k = threadIdx.x; k < N; k += blockDim.x) drho[(size_t)c * N + k] = f[k];
}

__global__ void __launch_bounds__(kThreads) step64_kernel(StepArgs a)
{
    extern __shared__ double sm[];
    __shared__ int s_cell;
    const DevTables &t = a.t;
    const int N = t.N, Np = t.Np;
    double *Wa = sm, *Wb = Wa + Np, *y = Wb + Np, *k1 = y + N, *k2 = k1 + N, *k3 = k2 + N,
           *k4 = k3 + N, *Y = k4 + N, *y1 = Y + N, *fl = y1 + N, *red = fl + N;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_cell = atomicAdd(a.counter, 1);
        __syncthreads();
        const int idx = s_cell;
        if (idx >= (a.wl.count ? *a.wl.count : t.n_cells)) break;
        const int c = a.wl.cells ? a.wl.cells[idx] : idx;
        const double t_span = a.wl.spans ? a.wl.spans[c] : a.t_span;   // this cell's span
        const double2 *Kc = a.K64 + (size_t)c * Np;
        double *rc = a.rho + (size_t)c * N;
        for (int k = threadIdx.x; k < N; k += blockDim.x) y[k] = rc[k];
        __syncthreads();
        double S = 0.0;                 // same summation order as a serial loop
        for (int k = 0; k < N; k++) S += y[k];
        const double atol = a.atol_rel * S;
        long long nacc = 0, nrej = 0;
        int status = CUDISC_OK;
        double h = 0.0;
        if (a.replay_h) {
            const long long nh = a.replay_n[c];
            const double *hs = a.replay_h + (size_t)c * a.replay_stride;
            for (long long s = 0; s < nh; s++) {
                const double hh = hs[s];
                rhs64(t, Kc, y, k1, Wa, Wb, fl);
                for (int k = threadIdx.x; k < N; k += blockDim.x) Y[k] = y[k] + hh * A21 * k1[k];
                __syncthreads();
                rhs64(t, Kc, Y, k2, Wa, Wb, fl);
                for (int k = threadIdx.x; k < N; k += blockDim.x) Y[k] = y[k] + hh * A32 * k2[k];
                __syncthreads();
                rhs64(t, Kc, Y, k3, Wa, Wb, fl);
                for (int k = threadIdx.x; k < N; k += blockDim.x)
                    y[k] = y[k] + hh * (B1 * k1[k] + B2 * k2[k] + B3 * k3[k]);
                __syncthreads();
            }
            nacc = nh;
        } else {
            rhs64(t, Kc, y, k1, Wa, Wb, fl);
            h = a.dt_cell ? a.dt_cell[c] : 0.0;
            if (!(h > 0.0)) {
                double q = INFINITY;
                for (int k = threadIdx.x; k < N; k += blockDim.x)
                    if (k1[k] != 0.0) q = fmin(q, (fabs(y[k]) + atol) / fabs(k1[k]));
                const double hmin = block_reduce(q, red, MinOp());
                h = isfinite(hmin) ? 0.1 * hmin : t_span;
                if (h > t_span) h = t_span;
            }
            double tt = 0.0;
            while (tt < t_span) {
                if (nacc + nrej >= a.max_steps) { status = CUDISC_EMAXSTEPS; break; }
                const bool last = (h >= t_span - tt);
                const double hs = last ? (t_span - tt) : h;
                for (int k = threadIdx.x; k < N; k += blockDim.x) Y[k] = y[k] + hs * A21 * k1[k];
                __syncthreads();
                rhs64(t, Kc, Y, k2, Wa, Wb, fl);
                for (int k = threadIdx.x; k < N; k += blockDim.x) Y[k] = y[k] + hs * A32 * k2[k];
                __syncthreads();
                rhs64(t, Kc, Y, k3, Wa, Wb, fl);
                for (int k = threadIdx.x; k < N; k += blockDim.x)
                    y1[k] = y[k] + hs * (B1 * k1[k] + B2 * k2[k] + B3 * k3[k]);
                __syncthreads();
                rhs64(t, Kc, y1, k4, Wa, Wb, fl);
                double E = 0.0, ymin = INFINITY, fin = 1.0;
                for (int k = threadIdx.x; k < N; k += blockDim.x) {
                    const double e = hs * (E1 * k1[k] + E2 * k2[k] + E3 * k3[k] + E4 * k4[k]);
                    const double sc = atol + a.rtol * fmax(fabs(y[k]), fabs(y1[k]));
                    const double r = (e == 0.0) ? 0.0 : fabs(e) / sc;   // an empty cell: no error
                    if (!isfinite(r) || !isfinite(y1[k])) fin = 0.0;
                    if (r > E) E = r;
                    if (y1[k] < ymin) ymin = y1[k];
                }
                E = block_reduce(E, red, MaxOp());
                ymin = block_reduce(ymin, red, MinOp());
                const bool finite = block_reduce(fin, red, MinOp()) > 0.5;
                if (finite && E <= 1.0 && ymin >= -atol) {
                    tt = last ? t_span : tt + hs;
                    for (int k = threadIdx.x; k < N; k += blockDim.x) { y[k] = y1[k]; k1[k] = k4[k]; }
                    if (threadIdx.x == 0 && a.rec_dt && nacc < a.rec_cap)
                        a.rec_dt[(size_t)c * a.rec_cap + nacc] = hs;
                    nacc++;
                    double fac = (E > 0.0) ? 0.9 * pow(E, -1.0 / 3.0) : 5.0;
                    fac = fmin(fmax(fac, 0.2), 5.0);
                    if (!(last && hs < h)) h = hs * fac;
                    __syncthreads();
                } else {
                    nrej++;
                    double fac;
                    if (!finite) fac = 0.2;
                    else if (E > 1.0) fac = fmax(0.9 * pow(E, -1.0 / 3.0), 0.2);
                    else fac = 0.5;
                    h = hs * fac;
                    if (h < 1e-14 * t_span) { status = finite ? CUDISC_EDTMIN : CUDISC_ENONFINITE; break; }
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < N; k += blockDim.x) rc[k] = y[k];
        if (threadIdx.x == 0) {
            double S1 = 0.0;
            for (int k = 0; k < N; k++) S1 += y[k];
            CellOut o;
            o.n_acc = nacc; o.n_rej = nrej; o.h_last = h;
            o.mass_err = S > 0.0 ? fabs(S1 / S - 1.0) : 0.0;
            o.status = status; o.pad = 0;
            a.out[c] = o;
            if (a.dt_cell && !a.replay_h) a.dt_cell[c] = h;
            if (a.rec_n) a.rec_n[c] = nacc;
            if (a.rec_status) a.rec_status[c] = status;
        }
    }
}

} // namespace

cudaError_t launch_rhs_fp64(const cudisc_coag_ctx *c, const double *rho, double *drho)
{
    const size_t smem = smem_doubles(c->N, c->Np) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(rhs64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (int c0 = 0; c0 < c->n_cells; c0 += (1 << 30)) {
        const int n = std::min(c->n_cells - c0, 1 << 30);
        rhs64_kernel<<<n, kThreads, smem, c->stream>>>(c0, c->tables(), c->d_K64, rho, drho);
    }
    return cudaGetLastError();
}

cudaError_t launch_step_fp64(const cudisc_coag_ctx *c, double *rho, double t_span,
                             double *dt_cell, const double *replay_h,
                             const long long *replay_n, long long replay_stride, WorkList wl)
{
    const size_t smem = smem_doubles(c->N, c->Np) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(step64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step64_kernel, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (c->p.max_sms > 0) n_sm = std::min(n_sm, c->p.max_sms);
    const int grid = std::max(1, std::min(c->n_cells, n_sm * per_sm));
    e = cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    StepArgs a;
    a.t = c->tables();
    a.K64 = c->d_K64;
    a.rho = rho;
    a.t_span = t_span;
    a.dt_cell = dt_cell;
    a.rtol = c->p.rtol;
    a.atol_rel = c->p.atol_rel;
    a.max_steps = c->p.max_substeps;
    a.replay_h = replay_h;
    a.replay_n = replay_n;
    a.replay_stride = replay_stride;
    a.out = c->d_out;
    a.counter = c->d_counter;
    a.rec_dt = c->rec_dt;
    a.rec_cap = c->rec_cap;
    a.rec_n = c->rec_n;
    a.rec_status = c->rec_status;
    a.wl = wl;
    step64_kernel<<<grid, kThreads, smem, c->stream>>>(a);
    return cudaGetLastError();
}

} // namespace cdc
