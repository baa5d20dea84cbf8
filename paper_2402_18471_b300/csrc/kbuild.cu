// Collision-kernel builder (Sec. 5): per-cell Stokes numbers and dust
// velocities, then per pair K_ij = pi (a_i + a_j)^2 dv_ij (Eq. kernel) with
// dv^2 = v_BM^2 + v_turb^2 + dv_lam^2 (Eqs. vbrown, OCVrel) and the
// fragmentation probability of Eq. (p_frag).  Output per pair: {K, K p_frag}.
//
// The FP32 builder feeds the mixed-precision contraction and is meant to be
// bound by the HBM writes of its output (8 B per pair).  It evaluates the
// Ormel & Cuzzi terms in a cancellation-free arrangement (see below).
#include <algorithm>
#include <cmath>

#include "coag_internal.h"
#include "oc07.cuh"

namespace cdc {
namespace {

struct KParams {
    double k_B, m_H, G, Mstar, mu, rho_m, sigma_H2, v_frag, kernel_const;
    int kernel_mode, frag_mode, vertical;
};

KParams kparams(const cudisc_coag_params &p)
{
    KParams k;
    k.k_B = p.k_B; k.m_H = p.m_H; k.G = p.G; k.Mstar = p.Mstar; k.mu = p.mu;
    k.rho_m = p.rho_m; k.sigma_H2 = p.sigma_H2; k.v_frag = p.v_frag;
    k.kernel_const = p.kernel_const; k.kernel_mode = p.kernel_mode; k.frag_mode = p.frag_mode;
    k.vertical = p.vertical;
    return k;
}

// One thread per (cell, bin): Epstein Stokes number (Eq. t_stop, St = t_s
// Omega), dust velocities (input or terminal drift and settling), and the
// per-bin parts of the Ormel & Cuzzi closed forms.  Vertically integrated
// kernel (Sec. 5.1): the cell is a radius at Z = 0, each grain a Gaussian
// layer of scale height h = H sqrt(alpha / (alpha + St)) settling at its
// terminal velocity at Z = h.
__global__ void __launch_bounds__(128) prep_kernel(
    int c0, KParams kp, int n_cells, int N, const double *__restrict__ a, const double *__restrict__ m,
    const double *__restrict__ rho_gas, const double *__restrict__ T,
    const double *__restrict__ alpha, const double *__restrict__ R,
    const double *__restrict__ Z, const double *__restrict__ eta,
    const double *__restrict__ v_dust, double *__restrict__ prep,
    float *__restrict__ prep32, CellScal *__restrict__ scal, float4 *__restrict__ scal32)
{
    const int c = c0 + blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells || k >= N) return;
    const double Tc = T[c], rg = rho_gas[c], Rc = R[c], Zc = kp.vertical ? 0.0 : Z[c], al = alpha[c];
    const double cs = sqrt(kp.k_B * Tc / (kp.mu * kp.m_H));
    const double vth = sqrt(8.0 / M_PI) * cs;
    const double r2 = Rc * Rc + Zc * Zc;
    const double Om = sqrt(kp.G * kp.Mstar / (r2 * sqrt(r2)));
    const double Om_mid = sqrt(kp.G * kp.Mstar / (Rc * Rc * Rc));
    const double nu_t = al * cs * (cs / Om_mid);
    const double nu_mol = 0.5 * vth * (kp.mu * kp.m_H / (rg * kp.sigma_H2));
    const double Re = nu_t / nu_mol;
    const double delta = 1.0 / sqrt(Re);
    const double St = kp.rho_m * a[k] / (rg * vth) * Om;
    const double hk = kp.vertical ? (cs / Om_mid) * sqrt(al / (al + St)) : 0.0;
    double vR, vphi, vZ;
    if (v_dust) {
        const size_t nc = (size_t)n_cells * N;
        vR = v_dust[(size_t)c * N + k];
        vphi = v_dust[nc + (size_t)c * N + k];
        vZ = v_dust[2 * nc + (size_t)c * N + k];
    } else {
        const double et = eta ? eta[c] : 0.0;
        const double vK = Om * Rc;
        vR = -2.0 * et * vK * St / (1.0 + St * St);
        vphi = -et * vK / (1.0 + St * St);
        vZ = -(kp.vertical ? hk : Zc) * Om * St / (1.0 + St);
    }
    const double g1 = St * St / (1.0 + St);      // St^2 / (t_L + St), t_L = 1
    const double g2 = St * St / (St + delta);    // St^2 / (t_eta + St)
    double *pr = prep + (size_t)c * PF_COUNT * N;
    float *pf = prep32 + (size_t)c * P3_COUNT * N;
    const double v[PF_COUNT] = {St, vR, vphi, vZ, g1, g2, hk};
#pragma unroll
    for (int f = 0; f < PF_COUNT; f++) pr[f * N + k] = v[f];
    const float vRh = (float)vR, vPh = (float)vphi, vZh = (float)vZ;
    const double Ss = fmin(fmax(1.6 * St, delta), 1.0);
    const float v32[P3_COUNT] = {(float)St, vRh, (float)(vR - vRh), vPh, (float)(vphi - vPh),
                                 vZh, (float)(vZ - vZh), (float)Ss, (float)(Ss - delta),
                                 (float)(1.0 - Ss), (float)(8.0 * kp.k_B * Tc / (M_PI * m[k])),
                                 (float)a[k], (float)m[k], (float)(2.0 * M_PI * hk * hk)};
#pragma unroll
    for (int f = 0; f < P3_COUNT; f++) pf[f * N + k] = v32[f];
    if (k == 0) {
        CellScal s;
        s.kT8pi = 8.0 * kp.k_B * Tc / M_PI;
        s.Vg2 = al * cs * cs;
        s.delta = delta;
        s.etavK = (eta ? eta[c] : 0.0) * Om * Rc;
        s.ZOm = Zc * Om;
        s.pad = 0.0;
        scal[c] = s;
        scal32[c] = make_float4((float)s.delta, (float)s.Vg2, (float)s.etavK, (float)s.ZOm);
    }
}

__global__ void __launch_bounds__(256) kbuild64_kernel(
    int c0, KParams kp, int n_cells, int N, int Np, const unsigned int *__restrict__ pij,
    const double *__restrict__ a, const double *__restrict__ minv,
    const double *__restrict__ m, const double *__restrict__ prep,
    const CellScal *__restrict__ scal, double2 *__restrict__ Kout)
{
    const int c = c0 + blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells || p >= Np) return;
    const unsigned int ij = pij[p];
    const int i = ij >> 16, j = ij & 0xffff;
    const double *pr = prep + (size_t)c * PF_COUNT * N;
    const CellScal s = scal[c];
    const double Si = pr[PF_ST * N + i], Sj = pr[PF_ST * N + j];
    const bool iw = Si >= Sj;
    const int i1 = iw ? i : j, i2 = iw ? j : i;
    const double V = vrel2_f64(pr[PF_ST * N + i1], pr[PF_ST * N + i2], pr[PF_G1 * N + i1],
                               pr[PF_G1 * N + i2], pr[PF_G2 * N + i1], pr[PF_G2 * N + i2], s.delta);
    const double vbm2 = s.kT8pi * (minv[i] + minv[j]);
    const double dR = pr[PF_VR * N + i] - pr[PF_VR * N + j];
    const double dP = pr[PF_VPHI * N + i] - pr[PF_VPHI * N + j];
    const double dZ = pr[PF_VZ * N + i] - pr[PF_VZ * N + j];
    const double dv = sqrt(vbm2 + s.Vg2 * V + (dR * dR + dP * dP + dZ * dZ));
    double K;
    if (kp.kernel_mode == CUDISC_KERNEL_CONSTANT) K = kp.kernel_const;
    else if (kp.kernel_mode == CUDISC_KERNEL_ADDITIVE) K = kp.kernel_const * (m[i] + m[j]);
    else { const double sa = a[i] + a[j]; K = M_PI * sa * sa * dv; }
    if (kp.vertical) {
        const double hi = pr[PF_H * N + i], hj = pr[PF_H * N + j];
        K /= sqrt(2.0 * M_PI * (hi * hi + hj * hj));
    }
    double pf;
    if (kp.frag_mode == CUDISC_FRAG_NONE) pf = 0.0;
    else if (kp.frag_mode == CUDISC_FRAG_ALL) pf = 1.0;
    else if (dv > 0.0) {
        const double q = kp.v_frag / dv;
        const double x = 1.5 * q * q;
        pf = (x + 1.0) * exp(-x);
    } else pf = 0.0;
    Kout[(size_t)c * Np + p] = make_double2(K, K * pf);
}

// Hardware approximations (flush-to-zero; a few ulp) for the FP32 builder.
__device__ __forceinline__ float rcp_ftz(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// e^-x = 2^(-x log2 e)
__device__ __forceinline__ float exp_neg_ftz(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x * -1.4426950408889634f));
    return r;
}

// Coagulation probability p_c = 1 - (1 + x) e^-x of Eq. (p_frag), accurate in
// FP32 also where p_frag rounds to 1: for x < 1 as x^2 g(x) with
//   g(x) = (1 - (1 + x) e^-x) / x^2 = e^-x sum_{m>=0} x^m / (m + 2)!,
// a smooth function with g(0) = 1/2, approximated on [0, 1] by its degree-6
// Chebyshev interpolant (interpolation error 6e-9 relative; evaluated by
// Horner in FP32 it is as accurate as the 13-term Taylor series it replaces,
// 1.6e-7); for x >= 1 from the closed form (p_c >= 0.26 there, no
// cancellation).  Given e = e^-x.  The coefficients are computed on the host
// (pcoag_poly).
struct PcoagPoly { float c[7]; };   // monomial coefficients, c[0] the constant term

__device__ __forceinline__ float pcoag_f32(float x, float e, const PcoagPoly &P)
{
    if (x >= 1.0f) return 1.0f - (1.0f + x) * e;
    float s = P.c[6];
#pragma unroll
    for (int k = 5; k >= 0; k--) s = s * x + P.c[k];
    return x * x * s;
}

// The degree-6 interpolant of g at the Chebyshev nodes of [0, 1], as monomial
// coefficients: g at the nodes from its all-positive series in FP64 (exact to
// rounding for x <= 1), then the Vandermonde system solved by Gaussian
// elimination with partial pivoting.
PcoagPoly pcoag_poly()
{
    constexpr int n = 7;
    double A[n][n + 1];
    for (int k = 0; k < n; k++) {
        const double x = 0.5 + 0.5 * std::cos((2 * k + 1) * M_PI / (2.0 * n));
        double s = 0.0, t = 0.5;
        for (int m = 0; m < 40; m++) { s += t; t *= x / (m + 3); }
        double p = 1.0;
        for (int j = 0; j < n; j++) { A[k][j] = p; p *= x; }
        A[k][n] = std::exp(-x) * s;
    }
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        for (int j = 0; j <= n; j++) std::swap(A[c][j], A[piv][j]);
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            const double f = A[r][c] / A[c][c];
            for (int j = c; j <= n; j++) A[r][j] -= f * A[c][j];
        }
    }
    PcoagPoly P;
    for (int j = 0; j < n; j++) P.c[j] = (float)(A[j][n] / A[j][j]);
    return P;
}

// Shared-memory fields of the FP32 builder, each [NR] (NR = N rounded up to
// 16, zero-padded so that four consecutive bins load as one 16-byte word):
// the prep fields P3_* up to P3_M, then 1/(1+St^2) and 1/(1+St), and, for the
// vertically integrated kernel only, 2 pi h^2.
enum { KB_INVA = P3_HH, KB_INVQ, KB_HH, KB_COUNT };

// FP32 builder in the blocked pair layout of the mixed contraction: slot
// q = 16 b + t is pair (blk_i[b], blk_j0[b] + t) and holds {K p_c, K p_f}
// (cell-major, see k32_index)
// (p_c = 1 - p_f, each accurate to a few ulp of itself, so that neither
// coagulation in a fragmentation-dominated cell nor fragmentation in a
// coagulation-dominated one is lost to rounding); slots past the diagonal
// hold zeros.  One CTA per kPosTile consecutive cells, kWarpsPerCell warps
// per cell, each taking a contiguous quarter of the cell's 4-slot groups
// (so that the grid is ~7 waves of the four CTAs an SM holds, not 1.7: the
// last, partial wave then costs ~1 % instead of ~15 %): the cells' per-bin
// fields are staged in shared memory once; each thread then produces four
// consecutive slots of a block (same i, j .. j+3) and writes them as two
// 16-byte chunks, a warp 1 KB of its cell's table per store pair.  The
// larger Stokes number of a pair (i, j <= i) is always St_i: St = rho_m a
// Omega / (rho_g v_th) rises with the bin's size.  Divisions, the square
// root and the exponential use the hardware approximations: K stays within
// 1e-6 and K p_frag within 1e-5 of FP64.
//   Physical = physical kernel and fragmentation probability (the other
//   modes are the closed-form test kernels); HasVdust = input velocities.
constexpr int kWarpsPerCell = 4;            // warps sharing one cell's table
constexpr int kPosTile = 8 / kWarpsPerCell; // cells per CTA of 256 threads

// words of shared memory per cell: the fields above (without KB_HH unless
// vertical) of NR each, rounded to 16 bytes
__host__ __device__ inline int kb_cell_stride(int NR, bool vertical)
{
    return ((vertical ? KB_COUNT : KB_HH) * NR + 3) / 4 * 4;
}

template <bool Physical, bool HasVdust>
__global__ void __launch_bounds__(256) kbuild32_kernel(
    float kc, float v_frag, int kernel_mode, int frag_mode, int vertical, int n_cells, int N, int NR,
    int n_slots, const int *__restrict__ blk_i, const int *__restrict__ blk_j0,
    const float *__restrict__ prep32, const float4 *__restrict__ scal32, PcoagPoly poly,
    float2 *__restrict__ Kout)
{
    extern __shared__ __align__(16) float f32s[];       // [kPosTile][cell stride]: [KB_COUNT][NR] each
    const int CS = kb_cell_stride(NR, vertical);
    const int cell0 = blockIdx.x * kPosTile;
    __shared__ int s_cell[kPosTile];
    if (threadIdx.x < kPosTile) {
        const int c = cell0 + (int)threadIdx.x;
        s_cell[threadIdx.x] = c < n_cells ? c : -1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kPosTile * P3_HH * NR; t += blockDim.x) {
        const int jc = t / (P3_HH * NR), r = t - jc * (P3_HH * NR);
        const int f = r / NR, k = r - f * NR;
        const int c = s_cell[jc];
        f32s[jc * CS + r] = (c >= 0 && k < N) ? prep32[((size_t)c * P3_COUNT + f) * N + k] : 0.0f;
    }
    if (vertical) {
        for (int t = threadIdx.x; t < kPosTile * NR; t += blockDim.x) {
            const int jc = t / NR, k = t - jc * NR;
            const int c = s_cell[jc];
            f32s[jc * CS + KB_HH * NR + k] = (c >= 0 && k < N) ? prep32[((size_t)c * P3_COUNT + P3_HH) * N + k] : 0.0f;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kPosTile * NR; t += blockDim.x) {
        const int jc = t / NR, k = t - jc * NR;
        float *F = f32s + jc * CS;
        const float S = F[P3_ST * NR + k];
        F[KB_INVA * NR + k] = 1.0f / (1.0f + S * S);
        F[KB_INVQ * NR + k] = 1.0f / (1.0f + S);
    }
    __syncthreads();
    const int jc = (threadIdx.x >> 5) / kWarpsPerCell;    // this warp's cell of the tile
    const int part = (threadIdx.x >> 5) % kWarpsPerCell;  // and its share of the cell's groups
    const int c = s_cell[jc];
    if (c < 0) return;
    const float *F = f32s + jc * CS;
    const float4 s4 = scal32[c];
    const float d = s4.x, Vg2 = s4.y, ev = s4.z, zo = s4.w;
    const float vf2 = 1.5f * v_frag * v_frag;
    const float *St = F + P3_ST * NR, *U = F + P3_U * NR, *Aa = F + P3_A * NR;
    const float *IA = F + KB_INVA * NR, *IQ = F + KB_INVQ * NR;
    float4 *dst = reinterpret_cast<float4 *>(Kout) + (size_t)c * (n_slots / 2);   // the cell's 2-pair chunks
    const int n_grp = n_slots / 4;
    const int g_end = (int)((long long)(part + 1) * n_grp / kWarpsPerCell);
    for (int g = (int)((long long)part * n_grp / kWarpsPerCell) + (threadIdx.x & 31); g < g_end; g += 32) {
        const int q0 = 4 * g;
        const int b = q0 >> 4;
        const int i = __ldg(blk_i + b);
        const int j0 = __ldg(blk_j0 + b) + (q0 & 15);
        if (j0 > i) {
            // all four slots lie past the diagonal
            dst[2 * g] = make_float4(0.f, 0.f, 0.f, 0.f);
            dst[2 * g + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        // bin i (the larger Stokes number)
        const float S1 = St[i], Ss = F[P3_SS * NR + i], Ssmd = F[P3_SSMD * NR + i];
        const float omSs = F[P3_OMSS * NR + i], Ui = U[i], ai = Aa[i], ia1 = IA[i], iq1 = IQ[i];
        const float P1 = S1 + Ss, Q1 = 1.0f + S1, R1 = S1 + d;
        const float sd = Ss + d, Sd = Ss * d, opSs = 1.0f + Ss;
        const float c1 = S1 * sd + Sd, PQ1 = P1 * Q1, PR1 = P1 * R1;
        // bins j0 .. j0+3
        const float4 S2v = *reinterpret_cast<const float4 *>(St + j0);
        const float4 Ujv = *reinterpret_cast<const float4 *>(U + j0);
        const float4 ajv = *reinterpret_cast<const float4 *>(Aa + j0);
        const float4 iav = *reinterpret_cast<const float4 *>(IA + j0);
        const float4 iqv = *reinterpret_cast<const float4 *>(IQ + j0);
        const float S2a[4] = {S2v.x, S2v.y, S2v.z, S2v.w};
        const float Uja[4] = {Ujv.x, Ujv.y, Ujv.z, Ujv.w};
        const float aja[4] = {ajv.x, ajv.y, ajv.z, ajv.w};
        const float iaa[4] = {iav.x, iav.y, iav.z, iav.w};
        const float iqa[4] = {iqv.x, iqv.y, iqv.z, iqv.w};
        float o[8];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int j = j0 + u;
            const float S2 = S2a[u];
            // Ormel & Cuzzi class I and II terms rearranged into sums and
            // products of non-negative factors (algebraically identical to
            // the closed forms).  In FP32 the literal forms cancel: with St*
            // clamped to Re^-1/2 and St1 = St2 class II is exactly zero but
            // leaves a residue ~1e-7 St^2/Re^-1/2, and for St >> 1 both
            // forms reduce to small differences of numbers near one.
            //   dVI  = (S1-S2)^2 (1-St*) [St*(S1+S2) + S1 S2 (1+St*)]
            //          / [(S1+S2)(St*+S1)(1+S1)(St*+S2)(1+S2)]
            //   dVII = (St*-d) sum_{s=S1,S2} [s (St*+d) + St* d] / [(s+St*)(s+d)]
            const float A = S1 + S2, P2 = S2 + Ss, Q2 = 1.0f + S2, R2 = S2 + d;
            const float dS = S1 - S2;
            const float nI = dS * dS * omSs * (Ss * A + S1 * S2 * opSs);
            const float dI = A * PQ1 * (P2 * Q2);
            const float PR2 = P2 * R2;
            const float nII = Ssmd * (c1 * PR2 + (S2 * sd + Sd) * PR1);
            const float dII = PR1 * PR2;
            const float V = fmaxf(nI * rcp_ftz(dI) + nII * rcp_ftz(dII), 0.0f);
            float dR, dP, dZ;
            if (HasVdust) {
                // input velocities: difference of FP32 hi/lo pairs
                dR = (F[P3_VRH * NR + i] - F[P3_VRH * NR + j]) + (F[P3_VRL * NR + i] - F[P3_VRL * NR + j]);
                dP = (F[P3_VPH * NR + i] - F[P3_VPH * NR + j]) + (F[P3_VPL * NR + i] - F[P3_VPL * NR + j]);
                dZ = (F[P3_VZH * NR + i] - F[P3_VZH * NR + j]) + (F[P3_VZL * NR + i] - F[P3_VZL * NR + j]);
            } else {
                // terminal velocities: differences factored through St_i - St_j
                //   v_R   = -2 eta v_K St/(1+St^2), v_phi = -eta v_K/(1+St^2),
                //   v_Z   = -Z Omega St/(1+St)
                const float rij = ia1 * iaa[u];
                dR = -2.0f * ev * dS * (1.0f - S1 * S2) * rij;
                dP = ev * dS * A * rij;
                dZ = -zo * dS * (iq1 * iqa[u]);
            }
            const float dv2 = (Ui + Uja[u]) + Vg2 * V + (dR * dR + dP * dP + dZ * dZ);
            const float rs = rsqrt_ftz(dv2);
            float K, pc, pf;
            if (Physical) {
                const float sa = ai + aja[u];
                K = 3.14159265358979f * sa * sa * (dv2 * rs);
                const float x = vf2 * (rs * rs);
                const float e = exp_neg_ftz(x);
                pf = (x + 1.0f) * e;
                pc = pcoag_f32(x, e, poly);
            } else {
                const float *Mm = F + P3_M * NR;
                if (kernel_mode == CUDISC_KERNEL_CONSTANT) K = kc;
                else if (kernel_mode == CUDISC_KERNEL_ADDITIVE) K = kc * (Mm[i] + Mm[j]);
                else { const float sa = ai + aja[u]; K = 3.14159265358979f * sa * sa * (dv2 * rs); }
                if (frag_mode == CUDISC_FRAG_NONE) { pf = 0.0f; pc = 1.0f; }
                else if (frag_mode == CUDISC_FRAG_ALL) { pf = 1.0f; pc = 0.0f; }
                else {
                    const float x = vf2 * (rs * rs);
                    const float e = exp_neg_ftz(x);
                    pf = (x + 1.0f) * e;
                    pc = pcoag_f32(x, e, poly);
                }
            }
            if (vertical) K *= rsqrt_ftz(F[KB_HH * NR + i] + F[KB_HH * NR + j]);
            const bool live = j <= i;
            o[2 * u] = live ? K * pc : 0.0f;
            o[2 * u + 1] = live ? K * pf : 0.0f;
        }
        dst[2 * g] = make_float4(o[0], o[1], o[2], o[3]);
        dst[2 * g + 1] = make_float4(o[4], o[5], o[6], o[7]);
    }
}

__global__ void get_kernel_kernel(int c0, int n_cells, int Np, int precision, int n_slots,
                                  const unsigned int *__restrict__ pij,
                                  const double2 *__restrict__ K64,
                                  const float2 *__restrict__ K32, double *__restrict__ K,
                                  double *__restrict__ KF)
{
    const int c = c0 + blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells || p >= Np) return;
    double k, kf;
    if (precision == CUDISC_FP64) {
        double2 v = K64[(size_t)c * Np + p];
        k = v.x; kf = v.y;
    } else {
        const unsigned int ij = pij[p];
        const int i = ij >> 16, j = ij & 0xffff;
        int row0 = 0;
        for (int r = 0; r < i; r++) row0 += (r + 16) >> 4;
        const int q = (row0 + (j >> 4)) * 16 + (j & 15);
        float2 v = K32[k32_index(c, q, n_slots)];   // {K p_c, K p_f}
        k = (double)v.x + (double)v.y; kf = v.y;
    }
    K[(size_t)c * Np + p] = k;
    KF[(size_t)c * Np + p] = kf;
}

} // namespace

cudaError_t launch_prep(const cudisc_coag_ctx *c)
{
    const cudisc_coag_params &p = c->p;
    for (int c0 = 0; c0 < c->n_cells; c0 += kMaxGridY) {
    dim3 grid((c->N + 127) / 128, std::min(kMaxGridY, c->n_cells - c0));
    prep_kernel<<<grid, 128, 0, c->stream>>>(c0, kparams(p), c->n_cells, c->N, c->d_a, c->d_m, p.rho_gas, p.T,
                                             p.alpha, p.R, p.Z, p.eta, p.v_dust, c->d_prep,
                                             c->d_prep32, c->d_scal, c->d_scal32);
    }
    return cudaGetLastError();
}

cudaError_t launch_kbuild(const cudisc_coag_ctx *c)
{
    const cudisc_coag_params &p = c->p;
    if (p.precision == CUDISC_FP64) {
        for (int c0 = 0; c0 < c->n_cells; c0 += kMaxGridY) {
        dim3 grid((c->Np + 255) / 256, std::min(kMaxGridY, c->n_cells - c0));
        kbuild64_kernel<<<grid, 256, 0, c->stream>>>(c0, kparams(p), c->n_cells, c->N, c->Np,
                                                     c->d_pair_ij, c->d_a, c->d_minv, c->d_m,
                                                     c->d_prep, c->d_scal, c->d_K64);
        }
    } else {
        const int n_slots = c->n_blk * kBlkPairs;
        const int NR = (c->N + 15) / 16 * 16;
        const size_t smem = (size_t)kPosTile * kb_cell_stride(NR, p.vertical != 0) * sizeof(float);
        const bool phys = p.kernel_mode == CUDISC_KERNEL_PHYSICAL && p.frag_mode == CUDISC_FRAG_PHYSICAL;
        // the vertically integrated kernel's settling velocities (each grain
        // at its own height) do not factor through St_i - St_j: take the
        // differences of the prep kernel's FP32 hi/lo velocity pairs
        const bool vd = p.v_dust != nullptr || p.vertical;
        auto kern = phys ? (vd ? kbuild32_kernel<true, true> : kbuild32_kernel<true, false>)
                         : (vd ? kbuild32_kernel<false, true> : kbuild32_kernel<false, false>);
        static const PcoagPoly poly = pcoag_poly();
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(c->n_cells + kPosTile - 1) / kPosTile, 256, smem, c->stream>>>(
            (float)p.kernel_const, (float)p.v_frag, p.kernel_mode, p.frag_mode, p.vertical, c->n_cells, c->N, NR,
            n_slots, c->d_blk_i, c->d_blk_j0, c->d_prep32, c->d_scal32, poly, c->d_K32);
    }
    return cudaGetLastError();
}

cudaError_t launch_get_kernel(const cudisc_coag_ctx *c, double *K, double *KF)
{
    for (int c0 = 0; c0 < c->n_cells; c0 += kMaxGridY) {
    dim3 grid((c->Np + 255) / 256, std::min(kMaxGridY, c->n_cells - c0));
    get_kernel_kernel<<<grid, 256, 0, c->stream>>>(c0, c->n_cells, c->Np, c->p.precision,
                                                   c->n_blk * kBlkPairs, c->d_pair_ij,
                                                   c->d_K64, c->d_K32, K, KF);
    }
    return cudaGetLastError();
}

} // namespace cdc
