// Discrete adjoint (vector-Jacobian product) of the coagulation step.
//
// The paper has no adjoint.  What is differentiated is the map the
// integrator applies: per cell, a fixed sequence of Bogacki-Shampine 3(2)
// steps (Sec. 5, last paragraph) with the step sizes frozen, applied to the
// right-hand side of Eq. (smol) written pair by pair:
//
//   f_k(y) = sum_p y_i y_j [ K_p a_pk + KF_p b_pk ],     KF_p = K_p p_frag,p,
//
// where a_pk holds the coagulation gain minus the loss of both grains and b_pk
// the remnant-plus-fragment gain minus the coagulation gain, per unit
// rho_i rho_j K (the host mapping tensor of Eqs. Cijk, Rijk, fragrem, Nijk).
// For a cotangent v the transpose is
//
//   Ga_p = sum_k a_pk v_k,   Gb_p = sum_k b_pk v_k + Mf_p Fv[l_p],
//   Fv[l] = sum_{k<=l} N_k(m^e_{l+1}) v_k,
//   ybar_i += (K_p Ga_p + KF_p Gb_p) y_j,  ybar_j += (K_p Ga_p + KF_p Gb_p) y_i,
//   Kbar_p = y_i y_j Ga_p,  KFbar_p = y_i y_j Gb_p,
//
// and, because K and KF depend only on the gas, the parameter gradients are
// alpha_bar = sum (Kbar dK/dalpha + KFbar dKF/dalpha) and
// v_frag_bar = sum KFbar dKF/dv_frag, accumulated over every transposed
// right-hand side.  The reverse BS3 step for y' = y + h (2/9 k1 + 1/3 k2 +
// 4/9 k3), k1 = f(y), k2 = f(y + h/2 k1), k3 = f(y + 3h/4 k2) is
//
//   w3 = J(Y3)^T (4h/9 lam);  w2 = J(Y2)^T (h/3 lam + 3h/4 w3);
//   lam <- lam + w3 + w2 + J(y)^T (2h/9 lam + h/2 w2).
//
// One CTA integrates one cell: a forward pass that stores the state every
// kSeg = 16 substeps, then per segment (last first) a forward recompute that
// keeps y, k1, k2 of each substep, and the reverse sweep over it.  The state
// is carried in units of the cell's initial dust mass S (x = rho / S, step
// h S), as in the mixed-precision integrator, so that products of small bin
// densities stay well inside the floating-point range.  The adjoint runs in
// FP64 for contexts of either precision (T = double; a mixed context supplies
// its FP32 kernel tables, widened), or, on request, in double-float (T = df,
// FP32 pairs of ~48 significant bits, see dfloat.cuh): the per-pair work of
// the forward recompute and of the transposed right-hand sides then runs on
// the FP32 pipes, while the N-vectors of the BS3 stages, the checkpoints and
// the parameter-gradient sums stay FP64.  Plain FP32 was measured and
// rejected for both halves:
//   - an FP32 forward recompute puts ~1e-4 of the largest gradient component
//     into a coagulation-fragmentation equilibrium, whose gradient is
//     sensitive to trajectory errors;
//   - FP32 transposed right-hand sides lose the gradient with respect to
//     large grains, which is a small difference of sweep-up sums (relative
//     error O(1) in some cells of a 64 x 32 x 80-bin disc).
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <vector>

#include "coag_internal.h"
#include "oc07.cuh"
#include "dfloat.cuh"

namespace cdc {

constexpr int kSeg = 16;            // checkpoint interval, substeps
constexpr int kVjpThreads = 256;
constexpr int kVecs64 = 8;          // FP64 N-vectors in shared memory per cell
constexpr int kVecsT = 4;           // T N-vectors

struct VjpState {
    bool tables = false;
    size_t tsz = 0;                 // sizeof(T)
    int n_ent = 0;                  // pair-major entries per pair
    void *Ntab = nullptr;                                                           // T
    unsigned short *pk = nullptr, *pl = nullptr;
    void *pa = nullptr, *pb = nullptr, *pmf = nullptr;                              // T
    void *ent_ab = nullptr, *fent_m = nullptr;      // forward gather coefficients, T ([nnz][2], [fnnz])
    int tprec = -1;                 // type of the tables: CUDISC_ADJOINT_FP64 or _DOUBLE_FLOAT
    int *pair_q = nullptr;
    void *kt = nullptr;             // [5][n_cells][Np] T: K, KF, dK/da, dKF/da, dKF/dvf
    double *ckpt = nullptr;         // [n_cells][seg_cap][N]
    long long seg_cap = 0;
    double *segbuf = nullptr;       // [n_cells][kSeg][3][N]
    double *vf_part = nullptr;      // [n_cells]
    int *cell_status = nullptr;     // [n_cells]
    double *rec_dt = nullptr;       // internal forward records
    long long *rec_n = nullptr;
    int *rec_st = nullptr;
    long long rec_cap = 0;
    double *rho_tmp = nullptr;
};

namespace {

template <typename T>
struct VjpArgs {
    int N, Np, n_cells, n_ent;
    const unsigned int *pij;
    const int *row, *ent_p, *frow, *fent_p;
    const T *ent_ab;                          // forward gather coefficients [nnz][2] (type T)
    const T *fent_m;
    const T *Ntab;                            // fragment spread [l][k] (type T), both directions
    const unsigned short *pk, *pl;
    const T *pa, *pb, *pmf;
    const T *K, *KF, *dKa, *dKFa, *dKFv;      // [n_cells][Np]
    const double *rho0, *hs, *w;
    const long long *n_h;
    long long stride;
    double *ckpt;
    long long seg_cap;
    double *segbuf;
    double *g_rho0, *g_alpha, *vf_part;
    int *cell_status;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T s)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += shfl_xor(s, o);
    return s;
}

// f = rhs(y) for one cell, y and the per-pair arithmetic in type T, f FP64.
// XK, XF: [Np] scratch; fT, fl: [N] scratch.
template <typename T>
__device__ void rhs_cell(const VjpArgs<T> &A, const T *__restrict__ Kc, const T *__restrict__ KFc,
                         const T *y, double *f, T *XK, T *XF, T *fT, T *fl)
{
    const int N = A.N, Np = A.Np;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int p = tid; p < Np; p += blockDim.x) {
        const unsigned int ij = __ldg(A.pij + p);
        const T x = y[ij >> 16] * y[ij & 0xffff];
        XK[p] = x * Kc[p];
        XF[p] = x * KFc[p];
    }
    __syncthreads();
    // per output bin k: gather its entries; rows N..2N-1 gather the fragment
    // mass per largest-fragment bin l
    for (int r = warp; r < 2 * N; r += nw) {
        T s = T(0);
        if (r < N) {
            const int e1 = __ldg(A.row + r + 1);
            for (int e = __ldg(A.row + r) + lane; e < e1; e += 32) {
                const int p = __ldg(A.ent_p + e);
                s += XK[p] * ldg(A.ent_ab + 2 * e) + XF[p] * ldg(A.ent_ab + 2 * e + 1);
            }
        } else {
            const int l = r - N;
            const int e1 = __ldg(A.frow + l + 1);
            for (int e = __ldg(A.frow + l) + lane; e < e1; e += 32)
                s += XF[__ldg(A.fent_p + e)] * ldg(A.fent_m + e);
        }
        s = warp_sum(s);
        if (lane == 0) {
            if (r < N) fT[r] = s;
            else fl[r - N] = s;
        }
    }
    __syncthreads();
    // spread the gathered fragment mass: f_k += sum_{l >= k} N_k(m^e_{l+1}) F_l
    for (int k = tid; k < N; k += blockDim.x) {
        T s = fT[k];
        for (int l = k; l < N; l++) s += ldg(A.Ntab + (size_t)l * N + k) * fl[l];
        f[k] = (double)s;
    }
    __syncthreads();
}

// out = J(x)^T v for one cell in type T, and the parameter-gradient terms of
// this transposed right-hand side added to accA / accV.  gq: [Np], Fv: [N].
template <typename T>
__device__ void rhs_vjp_cell(const VjpArgs<T> &A, const T *__restrict__ Kc, const T *__restrict__ KFc,
                             const T *__restrict__ dKa, const T *__restrict__ dKFa,
                             const T *__restrict__ dKFv, const T *x, const T *v, T *out, T *gq,
                             T *Fv, double &accA, double &accV)
{
    const int N = A.N, Np = A.Np;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int l = warp; l < N; l += nw) {
        T s = T(0);
        for (int k = lane; k <= l; k += 32) s += ldg(A.Ntab + (size_t)l * N + k) * v[k];
        s = warp_sum(s);
        if (lane == 0) Fv[l] = s;
    }
    __syncthreads();
    T tA = T(0), tV = T(0);
    for (int p = tid; p < Np; p += blockDim.x) {
        const unsigned int ij = __ldg(A.pij + p);
        const int i = ij >> 16, j = ij & 0xffff;
        T Ga = T(0), Gb = T(0);
        for (int e = 0; e < A.n_ent; e++) {
            const size_t o = (size_t)e * Np + p;
            const T vk = v[__ldg(A.pk + o)];
            Ga += ldg(A.pa + o) * vk;
            Gb += ldg(A.pb + o) * vk;
        }
        Gb += ldg(A.pmf + p) * Fv[__ldg(A.pl + p)];
        const T xx = x[i] * x[j];
        gq[p] = Kc[p] * Ga + KFc[p] * Gb;
        tA += xx * (Ga * dKa[p] + Gb * dKFa[p]);
        tV += xx * Gb * dKFv[p];
    }
    accA += (double)tA;
    accV += (double)tV;
    __syncthreads();
    // out_b = sum_{j<=b} gq(b,j) x_j + sum_{i>=b} gq(i,b) x_i
    for (int b = warp; b < N; b += nw) {
        T s = T(0);
        const int base = b * (b + 1) / 2;
        for (int j = lane; j <= b; j += 32) s += gq[base + j] * x[j];
        for (int i = b + lane; i < N; i += 32) s += gq[i * (i + 1) / 2 + b] * x[i];
        s = warp_sum(s);
        if (lane == 0) out[b] = s;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kVjpThreads) vjp_kernel(VjpArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *red = reinterpret_cast<double *>(smem_raw);          // 64 doubles
    T *XK = reinterpret_cast<T *>(red + 64);                      // [Np]; gq aliases it
    T *XF = XK + A.Np;
    double *v64 = reinterpret_cast<double *>(XF + A.Np);
    const int N = A.N, Np = A.Np;
    double *y = v64, *k1 = v64 + N, *k2 = v64 + 2 * N, *k3 = v64 + 3 * N, *st = v64 + 4 * N;
    double *lam = v64 + 6 * N, *bar = v64 + 7 * N;   // v64 + 5 N: unused
    T *vT = reinterpret_cast<T *>(v64 + kVecs64 * N);
    T *xs = vT, *v = vT + N, *out = vT + 2 * N, *Fv = vT + 3 * N;
    T *gq = XK;
    const int c = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const size_t cp = (size_t)c * Np;
    const T *Kc = A.K + cp, *KFc = A.KF + cp, *dKa = A.dKa + cp, *dKFa = A.dKFa + cp,
            *dKFv = A.dKFv + cp;
    const double *r0 = A.rho0 + (size_t)c * N;
    // f = rhs(yd): the input in type T (xs), out and Fv as the gather's scratch
    auto rhs = [&](const double *yd, double *f) {
        for (int k = tid; k < N; k += blockDim.x) xs[k] = (T)yd[k];
        __syncthreads();
        rhs_cell(A, Kc, KFc, xs, f, XK, XF, out, Fv);
    };

    // scale: the cell's initial dust mass
    if (warp == 0) {
        double s = 0.0;
        for (int k = lane; k < N; k += 32) s += r0[k];
        s = warp_sum(s);
        if (lane == 0) red[0] = (s > 0.0 && isfinite(s)) ? s : 1.0;
    }
    __syncthreads();
    const double S = red[0];
    for (int k = tid; k < N; k += blockDim.x) y[k] = r0[k] / S;
    __syncthreads();
    const long long n = A.n_h[c];
    const double *hc = A.hs + (size_t)c * A.stride;
    double *ck = A.ckpt + (size_t)c * A.seg_cap * N;
    double *sb = A.segbuf + (size_t)c * kSeg * 3 * N;

    // forward pass, checkpoint every kSeg substeps
    for (long long t = 0; t < n; t++) {
        const double h = hc[t] * S;
        if (t % kSeg == 0)
            for (int k = tid; k < N; k += blockDim.x) ck[(size_t)(t / kSeg) * N + k] = y[k];
        rhs(y, k1);
        for (int k = tid; k < N; k += blockDim.x) st[k] = y[k] + (0.5 * h) * k1[k];
        __syncthreads();
        rhs(st, k2);
        for (int k = tid; k < N; k += blockDim.x) st[k] = y[k] + (0.75 * h) * k2[k];
        __syncthreads();
        rhs(st, k3);
        for (int k = tid; k < N; k += blockDim.x)
            y[k] += h * ((2.0 / 9.0) * k1[k] + (1.0 / 3.0) * k2[k] + (4.0 / 9.0) * k3[k]);
        __syncthreads();
    }

    // reverse sweep
    for (int k = tid; k < N; k += blockDim.x) lam[k] = A.w[(size_t)c * N + k] * S;
    double accA = 0.0, accV = 0.0;
    const long long nseg = (n + kSeg - 1) / kSeg;
    for (long long s = nseg - 1; s >= 0; s--) {
        const long long t0 = s * kSeg, t1 = (t0 + kSeg < n) ? t0 + kSeg : n;
        for (int k = tid; k < N; k += blockDim.x) y[k] = ck[(size_t)s * N + k];
        __syncthreads();
        for (long long t = t0; t < t1; t++) {
            const double h = hc[t] * S;
            double *slot = sb + (size_t)(t - t0) * 3 * N;
            rhs(y, k1);
            for (int k = tid; k < N; k += blockDim.x) {
                slot[k] = y[k];
                slot[N + k] = k1[k];
                st[k] = y[k] + (0.5 * h) * k1[k];
            }
            __syncthreads();
            rhs(st, k2);
            for (int k = tid; k < N; k += blockDim.x) slot[2 * N + k] = k2[k];
            if (t + 1 < t1) {
                for (int k = tid; k < N; k += blockDim.x) st[k] = y[k] + (0.75 * h) * k2[k];
                __syncthreads();
                rhs(st, k3);
                for (int k = tid; k < N; k += blockDim.x)
                    y[k] += h * ((2.0 / 9.0) * k1[k] + (1.0 / 3.0) * k2[k] + (4.0 / 9.0) * k3[k]);
            }
            __syncthreads();
        }
        for (long long t = t1 - 1; t >= t0; t--) {
            const double h = hc[t] * S;
            const double *slot = sb + (size_t)(t - t0) * 3 * N;
            // The transposed right-hand side is linear in its cotangent: run it
            // on lam / sig with sig a power of two near max |lam| (exact in
            // both directions), so that products such as K_p Ga_p stay far
            // from the range limits whatever the loss weights' units.
            if (warp == 0) {
                double mx = 0.0;
                for (int k = lane; k < N; k += 32) mx = fmax(mx, fabs(lam[k]));
                for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) red[1] = (mx > 0.0 && isfinite(mx)) ? exp2(floor(log2(mx))) : 1.0;
            }
            __syncthreads();
            const double sig = red[1], isig = 1.0 / sig;
            // Y3 = y + 3h/4 k2: w3 = J(Y3)^T (4h/9 lam)
            for (int k = tid; k < N; k += blockDim.x) {
                y[k] = slot[k];
                k1[k] = slot[N + k];
                xs[k] = (T)(slot[k] + (0.75 * h) * slot[2 * N + k]);
                v[k] = (T)((h * (4.0 / 9.0)) * (lam[k] * isig));
            }
            __syncthreads();
            double aA = 0.0, aV = 0.0;
            rhs_vjp_cell(A, Kc, KFc, dKa, dKFa, dKFv, xs, v, out, gq, Fv, aA, aV);
            // Y2 = y + h/2 k1: w2 = J(Y2)^T (h/3 lam + 3h/4 w3)   (all / sig)
            for (int k = tid; k < N; k += blockDim.x) {
                const double w3 = (double)out[k];
                bar[k] = lam[k] + w3 * sig;
                v[k] = (T)((h * (1.0 / 3.0)) * (lam[k] * isig) + (0.75 * h) * w3);
                xs[k] = (T)(y[k] + (0.5 * h) * k1[k]);
            }
            __syncthreads();
            rhs_vjp_cell(A, Kc, KFc, dKa, dKFa, dKFv, xs, v, out, gq, Fv, aA, aV);
            // y: w1 = J(y)^T (2h/9 lam + h/2 w2)   (all / sig)
            for (int k = tid; k < N; k += blockDim.x) {
                const double w2 = (double)out[k];
                bar[k] += w2 * sig;
                v[k] = (T)((h * (2.0 / 9.0)) * (lam[k] * isig) + (0.5 * h) * w2);
                xs[k] = (T)y[k];
            }
            __syncthreads();
            rhs_vjp_cell(A, Kc, KFc, dKa, dKFa, dKFv, xs, v, out, gq, Fv, aA, aV);
            for (int k = tid; k < N; k += blockDim.x) lam[k] = bar[k] + (double)out[k] * sig;
            accA += aA * sig;
            accV += aV * sig;
            __syncthreads();
        }
    }

    // outputs: d/d rho0 = lam_x / S; scalar gradients reduced over the block
    bool bad = false;
    for (int k = tid; k < N; k += blockDim.x) {
        const double g = lam[k] / S;
        bad |= !isfinite(g);
        A.g_rho0[(size_t)c * N + k] = g;
    }
    accA = warp_sum(accA);
    accV = warp_sum(accV);
    const int any_bad = __syncthreads_or(bad);
    if (lane == 0) { red[8 + warp] = accA; red[40 + warp] = accV; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < nw; w++) { a += red[8 + w]; b += red[40 + w]; }
        if (A.g_alpha) A.g_alpha[c] = a;
        A.vf_part[c] = b;
        A.cell_status[c] = (any_bad || !isfinite(a) || !isfinite(b)) ? CUDISC_ENONFINITE : CUDISC_OK;
    }
}

// Per-pair K, K p_frag and their derivatives with respect to alpha and
// v_frag, in FP64 from the prep fields; written in the adjoint's type T in
// packed pair order.  K and KF are the values the context's forward uses.
//   dv^2 = v_BM^2 + alpha c_s^2 V(St_i, St_j, d) + dv_lam^2,  d = Re^-1/2 ~ alpha^-1/2
//   d(dv^2)/d alpha = c_s^2 (V - d/2 dV/dd)
//   K = pi (a_i + a_j)^2 dv  ->  dK/d alpha = pi (a_i + a_j)^2 d(dv)/d alpha
//   p_frag = (1 + x) e^-x, x = 1.5 (v_f / dv)^2:
//       dp/d dv = 2 x^2 e^-x / dv,   dp/d v_f = -2 x^2 e^-x / v_f
template <typename T>
__global__ void __launch_bounds__(256) kderiv_kernel(
    int c0, int n_cells, int N, int Np, int kernel_mode, int frag_mode, double v_frag, int vertical,
    int has_vdust, const unsigned int *__restrict__ pij, const int *__restrict__ pair_q, int n_slots,
    const double *__restrict__ a, const double *__restrict__ minv,
    const double *__restrict__ prep, const CellScal *__restrict__ scal,
    const double *__restrict__ alpha, const double2 *__restrict__ K64,
    const float2 *__restrict__ K32, T *__restrict__ kt)
{
    const int c = c0 + blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells || p >= Np) return;
    const unsigned int ij = pij[p];
    const int i = ij >> 16, j = ij & 0xffff;
    double K, KF;
    if (K64) { const double2 v = K64[(size_t)c * Np + p]; K = v.x; KF = v.y; }
    else {   // mixed tables hold {K p_c, K p_f}
        const float2 v = K32[k32_index(c, pair_q[p], n_slots)];
        K = (double)v.x + (double)v.y;
        KF = v.y;
    }
    const double *pr = prep + (size_t)c * PF_COUNT * N;
    const CellScal s = scal[c];
    const double Si = pr[PF_ST * N + i], Sj = pr[PF_ST * N + j];
    const int i1 = Si >= Sj ? i : j, i2 = Si >= Sj ? j : i;
    const double S1 = pr[PF_ST * N + i1], S2 = pr[PF_ST * N + i2];
    const double V = vrel2_f64(S1, S2, pr[PF_G1 * N + i1], pr[PF_G1 * N + i2], pr[PF_G2 * N + i1],
                               pr[PF_G2 * N + i2], s.delta);
    const double dR = pr[PF_VR * N + i] - pr[PF_VR * N + j];
    const double dP = pr[PF_VPHI * N + i] - pr[PF_VPHI * N + j];
    const double dZ = pr[PF_VZ * N + i] - pr[PF_VZ * N + j];
    const double dv = sqrt(s.kT8pi * (minv[i] + minv[j]) + s.Vg2 * V + (dR * dR + dP * dP + dZ * dZ));
    const double al = alpha[c];
    const double cs2 = s.Vg2 / al;
    double ddv2_da = cs2 * (V - 0.5 * s.delta * dvrel2_dd_f64(S1, S2, s.delta));
    // vertically integrated kernel: dh/dalpha = h g, g = St / (2 alpha
    // (alpha + St)); the settling velocities (at Z = h) scale with h, and the
    // layer factor f = (2 pi (h_i^2 + h_j^2))^-1/2 has d ln f / dalpha =
    // -(h_i^2 g_i + h_j^2 g_j) / (h_i^2 + h_j^2)
    double gi = 0.0, gj = 0.0;
    if (vertical) {
        gi = Si / (2.0 * al * (al + Si));
        gj = Sj / (2.0 * al * (al + Sj));
        if (!has_vdust) ddv2_da += 2.0 * dZ * (pr[PF_VZ * N + i] * gi - pr[PF_VZ * N + j] * gj);
    }
    const double ddv_da = dv > 0.0 ? ddv2_da / (2.0 * dv) : 0.0;
    double dK_da = 0.0;
    if (kernel_mode == CUDISC_KERNEL_PHYSICAL) {
        const double sa = a[i] + a[j];
        dK_da = M_PI * sa * sa * ddv_da;
    }
    if (vertical) {
        const double hi = pr[PF_H * N + i], hj = pr[PF_H * N + j];
        const double hi2 = hi * hi, hj2 = hj * hj;
        const double f = 1.0 / sqrt(2.0 * M_PI * (hi2 + hj2));
        dK_da = f * dK_da - K * (hi2 * gi + hj2 * gj) / (hi2 + hj2);   // K includes f
    }
    double pf = 0.0, dpf_ddv = 0.0, dpf_dvf = 0.0;
    if (frag_mode == CUDISC_FRAG_ALL) pf = 1.0;
    else if (frag_mode == CUDISC_FRAG_PHYSICAL && dv > 0.0) {
        const double q = v_frag / dv;
        const double x = 1.5 * q * q;
        const double e = exp(-x);
        pf = (1.0 + x) * e;
        dpf_ddv = 2.0 * x * x * e / dv;
        dpf_dvf = -2.0 * x * x * e / v_frag;
    }
    const T o[5] = {(T)K, (T)KF, (T)dK_da, (T)(pf * dK_da + K * dpf_ddv * ddv_da),
                    (T)(K * dpf_dvf)};
    const size_t plane = (size_t)n_cells * Np;
#pragma unroll
    for (int f = 0; f < 5; f++) kt[f * plane + (size_t)c * Np + p] = o[f];
}

__global__ void vf_reduce_kernel(int n_cells, const double *__restrict__ part,
                                 const int *__restrict__ status, double *__restrict__ out,
                                 int *__restrict__ worst)
{
    __shared__ double sh[32];
    __shared__ int shw[32];
    double s = 0.0;
    int wst = 0;
    for (int c = threadIdx.x; c < n_cells; c += blockDim.x) {
        s += part[c];
        wst = max(wst, status[c]);
    }
    s = warp_sum(s);
    for (int o = 16; o > 0; o >>= 1) wst = max(wst, __shfl_xor_sync(0xffffffffu, wst, o));
    if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5] = s; shw[threadIdx.x >> 5] = wst; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        int w = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) { t += sh[k]; w = max(w, shw[k]); }
        if (out) *out = t;
        *worst = w;
    }
}

template <class V>
cudaError_t upload_vec(V **dst, const std::vector<V> &src, cudaStream_t st)
{
    cudaError_t e = cudaMalloc((void **)dst, std::max<size_t>(src.size(), 1) * sizeof(V));
    if (e != cudaSuccess || src.empty()) return e;
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

template <class V>
cudaError_t download_vec(std::vector<V> &dst, const V *src, size_t n, cudaStream_t st)
{
    dst.resize(n);
    if (!n) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst.data(), src, n * sizeof(V), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

template <typename T>
cudaError_t upload_as(void **dst, const std::vector<double> &src, cudaStream_t st)
{
    std::vector<T> t(src.begin(), src.end());
    T *d = nullptr;
    cudaError_t e = upload_vec(&d, t, st);
    *dst = d;
    return e;
}

template <typename T>
cudaError_t build_tables_t(cudisc_coag_ctx *c, VjpState *S)
{
    const int N = c->N, Np = c->Np;
    cudaStream_t st = c->stream;
    // the forward gather tables as the context built them (FP64, host
    // double-double coefficients), read back once
    std::vector<int> row, ent_p, frow, fent_p;
    std::vector<double2> ent_ab;
    std::vector<double> fent_m, Ntab;
    cudaError_t e;
    if ((e = download_vec(row, c->d_row, N + 1, st)) != cudaSuccess) return e;
    if ((e = download_vec(frow, c->d_frow, N + 1, st)) != cudaSuccess) return e;
    if ((e = download_vec(ent_p, c->d_ent_p, row[N], st)) != cudaSuccess) return e;
    if ((e = download_vec(ent_ab, c->d_ent_ab, row[N], st)) != cudaSuccess) return e;
    if ((e = download_vec(fent_p, c->d_fent_p, frow[N], st)) != cudaSuccess) return e;
    if ((e = download_vec(fent_m, c->d_fent_m, frow[N], st)) != cudaSuccess) return e;
    if ((e = download_vec(Ntab, c->d_Ntab, (size_t)N * N, st)) != cudaSuccess) return e;

    // pair-major transpose of the gather: per pair its (bin, a, b) entries
    std::vector<std::vector<int>> by_pair(Np);
    for (int k = 0; k < N; k++)
        for (int q = row[k]; q < row[k + 1]; q++) by_pair[ent_p[q]].push_back(q);
    int n_ent = 1;
    for (auto &v : by_pair) n_ent = std::max<int>(n_ent, (int)v.size());
    std::vector<unsigned short> pk((size_t)n_ent * Np, 0), pl(Np, 0);
    std::vector<double> pa((size_t)n_ent * Np, 0.0), pb((size_t)n_ent * Np, 0.0), pmf(Np, 0.0);
    std::vector<int> bin_of(row[N]);
    for (int k = 0; k < N; k++)
        for (int q = row[k]; q < row[k + 1]; q++) bin_of[q] = k;
    for (int p = 0; p < Np; p++)
        for (size_t t = 0; t < by_pair[p].size(); t++) {
            const int q = by_pair[p][t];
            pk[t * Np + p] = (unsigned short)bin_of[q];
            pa[t * Np + p] = ent_ab[q].x;
            pb[t * Np + p] = ent_ab[q].y;
        }
    for (int l = 0; l < N; l++)
        for (int q = frow[l]; q < frow[l + 1]; q++) {
            pmf[fent_p[q]] = fent_m[q];
            pl[fent_p[q]] = (unsigned short)l;
        }
    // mixed contexts keep K in the blocked pair layout of the contraction
    std::vector<int> pq(Np, 0);
    for (int i = 0, row0 = 0; i < N; row0 += (i + kBlkPairs) / kBlkPairs, i++)
        for (int j = 0; j <= i; j++)
            pq[i * (i + 1) / 2 + j] = (row0 + j / kBlkPairs) * kBlkPairs + j % kBlkPairs;

    S->n_ent = n_ent;
    S->tsz = sizeof(T);
    S->tprec = std::is_same<T, df>::value ? CUDISC_ADJOINT_DOUBLE_FLOAT : CUDISC_ADJOINT_FP64;
    std::vector<double> ab2(2 * ent_ab.size());
    for (size_t q = 0; q < ent_ab.size(); q++) { ab2[2 * q] = ent_ab[q].x; ab2[2 * q + 1] = ent_ab[q].y; }
    if ((e = upload_as<T>(&S->ent_ab, ab2, st)) != cudaSuccess) return e;
    if ((e = upload_as<T>(&S->fent_m, fent_m, st)) != cudaSuccess) return e;
    if ((e = upload_as<T>(&S->Ntab, Ntab, st)) != cudaSuccess) return e;
    if ((e = upload_as<T>(&S->pa, pa, st)) != cudaSuccess) return e;
    if ((e = upload_as<T>(&S->pb, pb, st)) != cudaSuccess) return e;
    if ((e = upload_as<T>(&S->pmf, pmf, st)) != cudaSuccess) return e;
    if ((e = upload_vec(&S->pk, pk, st)) != cudaSuccess) return e;
    if ((e = upload_vec(&S->pl, pl, st)) != cudaSuccess) return e;
    if ((e = upload_vec(&S->pair_q, pq, st)) != cudaSuccess) return e;
    const size_t nc = (size_t)c->n_cells;
    if ((e = cudaMalloc(&S->kt, 5 * nc * Np * sizeof(T))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&S->segbuf, nc * kSeg * 3 * N * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&S->vf_part, nc * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&S->cell_status, (nc + 1) * sizeof(int))) != cudaSuccess) return e;
    S->tables = true;
    return cudaSuccess;
}

template <typename T>
size_t vjp_smem(int N, int Np)
{
    return (64 + 2 * (size_t)Np + (size_t)kVecs64 * N) * sizeof(double) + (size_t)kVecsT * N * sizeof(T);
}

template <typename T>
cudaError_t launch_t(cudisc_coag_ctx *c, VjpState *S, const double *rho0, const double *hs,
                     const long long *n_h, long long stride, const double *w, double *g_rho0,
                     double *g_alpha, double *g_vf)
{
    const cudisc_coag_params &p = c->p;
    const int N = c->N, Np = c->Np;
    const size_t plane = (size_t)c->n_cells * Np;
    T *kt = static_cast<T *>(S->kt);
    for (int c0 = 0; c0 < c->n_cells; c0 += kMaxGridY) {
        dim3 grid((Np + 255) / 256, std::min(kMaxGridY, c->n_cells - c0));
        kderiv_kernel<T><<<grid, 256, 0, c->stream>>>(
            c0, c->n_cells, N, Np, p.kernel_mode, p.frag_mode, p.v_frag, p.vertical, p.v_dust != nullptr,
            c->d_pair_ij, S->pair_q,
            c->n_blk * kBlkPairs, c->d_a, c->d_minv, c->d_prep, c->d_scal, p.alpha, c->d_K64,
            c->d_K32, kt);
    }
    VjpArgs<T> A;
    A.N = N; A.Np = Np; A.n_cells = c->n_cells; A.n_ent = S->n_ent;
    A.pij = c->d_pair_ij;
    A.row = c->d_row; A.ent_p = c->d_ent_p; A.frow = c->d_frow; A.fent_p = c->d_fent_p;
    A.ent_ab = static_cast<const T *>(S->ent_ab); A.fent_m = static_cast<const T *>(S->fent_m);
    A.Ntab = static_cast<const T *>(S->Ntab);
    A.pk = S->pk; A.pl = S->pl;
    A.pa = static_cast<const T *>(S->pa); A.pb = static_cast<const T *>(S->pb);
    A.pmf = static_cast<const T *>(S->pmf);
    A.K = kt; A.KF = kt + plane; A.dKa = kt + 2 * plane; A.dKFa = kt + 3 * plane;
    A.dKFv = kt + 4 * plane;
    A.rho0 = rho0; A.hs = hs; A.w = w; A.n_h = n_h; A.stride = stride;
    A.ckpt = S->ckpt; A.seg_cap = S->seg_cap;
    A.segbuf = S->segbuf;
    A.g_rho0 = g_rho0; A.g_alpha = g_alpha; A.vf_part = S->vf_part;
    A.cell_status = S->cell_status;
    const size_t smem = vjp_smem<T>(N, Np);
    cudaError_t e = cudaFuncSetAttribute(vjp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    vjp_kernel<T><<<c->n_cells, kVjpThreads, smem, c->stream>>>(A);
    vf_reduce_kernel<<<1, 256, 0, c->stream>>>(c->n_cells, S->vf_part, S->cell_status, g_vf,
                                               S->cell_status + c->n_cells);
    return cudaGetLastError();
}

// the tables built for one arithmetic type (kept: checkpoints and records)
void free_tables(VjpState *S)
{
    void *ptrs[] = {S->Ntab, S->pk, S->pl, S->pa, S->pb, S->pmf, S->ent_ab, S->fent_m,
                    S->pair_q, S->kt, S->segbuf, S->vf_part, S->cell_status};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    S->Ntab = S->pa = S->pb = S->pmf = S->ent_ab = S->fent_m = S->kt = nullptr;
    S->pk = S->pl = nullptr;
    S->pair_q = S->cell_status = nullptr;
    S->segbuf = S->vf_part = nullptr;
    S->tables = false;
    S->tprec = -1;
}

} // namespace

bool vjp_fits(const cudisc_coag_ctx *c)
{
    static_assert(sizeof(df) == sizeof(double), "both adjoint types share one shared-memory layout");
    return vjp_smem<double>(c->N, c->Np) <= 232448;
}

cudaError_t vjp_prepare(cudisc_coag_ctx *c, long long max_steps)
{
    if (!c->vjp) c->vjp = new VjpState();
    VjpState *S = c->vjp;
    cudaError_t e = cudaSuccess;
    if (S->tables && S->tprec != c->adj_prec) free_tables(S);
    if (!S->tables) {
        e = c->adj_prec == CUDISC_ADJOINT_DOUBLE_FLOAT ? build_tables_t<df>(c, S) : build_tables_t<double>(c, S);
        if (e != cudaSuccess) return e;
    }
    const long long need = std::max<long long>(1, (max_steps + kSeg - 1) / kSeg);
    if (need > S->seg_cap) {
        if (S->ckpt) cudaFree(S->ckpt);
        S->ckpt = nullptr;
        S->seg_cap = 0;
        e = cudaMalloc(&S->ckpt, (size_t)c->n_cells * need * c->N * sizeof(double));
        if (e != cudaSuccess) return e;
        S->seg_cap = need;
    }
    return cudaSuccess;
}

cudaError_t vjp_records(cudisc_coag_ctx *c, long long cap, double **dt, long long **n, int **status,
                        double **rho_tmp)
{
    if (!c->vjp) c->vjp = new VjpState();
    VjpState *S = c->vjp;
    cudaError_t e;
    if (cap > S->rec_cap) {
        if (S->rec_dt) cudaFree(S->rec_dt);
        S->rec_dt = nullptr;
        S->rec_cap = 0;
        if ((e = cudaMalloc(&S->rec_dt, (size_t)c->n_cells * cap * sizeof(double))) != cudaSuccess)
            return e;
        S->rec_cap = cap;
    }
    if (!S->rec_n && (e = cudaMalloc(&S->rec_n, c->n_cells * sizeof(long long))) != cudaSuccess) return e;
    if (!S->rec_st && (e = cudaMalloc(&S->rec_st, c->n_cells * sizeof(int))) != cudaSuccess) return e;
    if (!S->rho_tmp &&
        (e = cudaMalloc(&S->rho_tmp, (size_t)c->n_cells * c->N * sizeof(double))) != cudaSuccess)
        return e;
    *dt = S->rec_dt;
    *n = S->rec_n;
    *status = S->rec_st;
    *rho_tmp = S->rho_tmp;
    return cudaSuccess;
}

cudaError_t launch_vjp(cudisc_coag_ctx *c, const double *rho0, const double *hs,
                       const long long *n_h, long long stride, const double *w, double *g_rho0,
                       double *g_alpha, double *g_vf)
{
    if (c->vjp->tprec == CUDISC_ADJOINT_DOUBLE_FLOAT)
        return launch_t<df>(c, c->vjp, rho0, hs, n_h, stride, w, g_rho0, g_alpha, g_vf);
    return launch_t<double>(c, c->vjp, rho0, hs, n_h, stride, w, g_rho0, g_alpha, g_vf);
}

cudaError_t vjp_worst_status(const cudisc_coag_ctx *c, int *worst)
{
    return cudaMemcpy(worst, c->vjp->cell_status + c->n_cells, sizeof(int), cudaMemcpyDeviceToHost);
}

void vjp_free(cudisc_coag_ctx *c)
{
    VjpState *S = c->vjp;
    if (!S) return;
    void *ptrs[] = {S->Ntab, S->pk, S->pl, S->pa, S->pb, S->pmf,
                    S->pair_q, S->kt, S->ckpt, S->segbuf, S->vf_part, S->cell_status, S->rec_dt,
                    S->rec_n, S->rec_st, S->rho_tmp};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (S->ent_ab) cudaFree(S->ent_ab);
    if (S->fent_m) cudaFree(S->fent_m);
    delete S;
    c->vjp = nullptr;
}

} // namespace cdc
