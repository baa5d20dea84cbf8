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
    int kernel_mode, frag_mode;
};

KParams kparams(const cudisc_coag_params &p)
{
    KParams k;
    k.k_B = p.k_B; k.m_H = p.m_H; k.G = p.G; k.Mstar = p.Mstar; k.mu = p.mu;
    k.rho_m = p.rho_m; k.sigma_H2 = p.sigma_H2; k.v_frag = p.v_frag;
    k.kernel_const = p.kernel_const; k.kernel_mode = p.kernel_mode; k.frag_mode = p.frag_mode;
    return k;
}

// One thread per (cell, bin): Epstein Stokes number (Eq. t_stop, St = t_s
// Omega), dust velocities (input or terminal drift and settling), and the
// per-bin parts of the Ormel & Cuzzi closed forms.
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
    const double Tc = T[c], rg = rho_gas[c], Rc = R[c], Zc = Z[c], al = alpha[c];
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
        vZ = -Zc * Om * St / (1.0 + St);
    }
    const double g1 = St * St / (1.0 + St);      // St^2 / (t_L + St), t_L = 1
    const double g2 = St * St / (St + delta);    // St^2 / (t_eta + St)
    double *pr = prep + (size_t)c * PF_COUNT * N;
    float *pf = prep32 + (size_t)c * P3_COUNT * N;
    const double v[PF_COUNT] = {St, vR, vphi, vZ, g1, g2};
#pragma unroll
    for (int f = 0; f < PF_COUNT; f++) pr[f * N + k] = v[f];
    const float vRh = (float)vR, vPh = (float)vphi, vZh = (float)vZ;
    const double Ss = fmin(fmax(1.6 * St, delta), 1.0);
    const float v32[P3_COUNT] = {(float)St, vRh, (float)(vR - vRh), vPh, (float)(vphi - vPh),
                                 vZh, (float)(vZ - vZh), (float)Ss, (float)(Ss - delta),
                                 (float)(1.0 - Ss), (float)(8.0 * kp.k_B * Tc / (M_PI * m[k])),
                                 (float)a[k], (float)m[k]};
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

// FP32 builder in the blocked pair layout of the mixed contraction: slot
// q = 16 b + t is pair (blk_i[b], blk_j0[b] + t); slots past the diagonal
// hold zeros.
__global__ void __launch_bounds__(256) kbuild32_kernel(
    int c0, float kc, float v_frag, int kernel_mode, int frag_mode, int has_vdust, int n_cells,
    int N, int n_slots,
    const int *__restrict__ blk_i, const int *__restrict__ blk_j0,
    const double *__restrict__ a, const double *__restrict__ minv,
    const double *__restrict__ m, const float *__restrict__ prep32,
    const float4 *__restrict__ scal32, float2 *__restrict__ Kout)
{
    const int c = c0 + blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells || q >= n_slots) return;
    const int b = q >> 4;
    const int i = blk_i[b];
    const int j = blk_j0[b] + (q & 15);
    float2 out = make_float2(0.f, 0.f);
    if (j <= i) {
        const float *pr = prep32 + (size_t)c * P3_COUNT * N;
        const float4 s4 = scal32[c];
        const float d = s4.x, Vg2 = s4.y;
        const float Si = pr[P3_ST * N + i], Sj = pr[P3_ST * N + j];
        float S1 = Si, S2 = Sj;
        int i1 = i;
        if (S2 > S1) { float t = S1; S1 = S2; S2 = t; i1 = j; }
        const float Ss = pr[P3_SS * N + i1];
        const float Ssmd = pr[P3_SSMD * N + i1], omSs = pr[P3_OMSS * N + i1];
        // Ormel & Cuzzi class I and II terms rearranged into sums and
        // products of non-negative factors (algebraically identical to the
        // closed forms).  In FP32 the literal forms cancel: with St* clamped
        // to Re^-1/2 and St1 = St2 class II is exactly zero but leaves a
        // residue ~1e-7 St^2/Re^-1/2, and for St >> 1 both forms reduce to
        // small differences of numbers near one.
        //   dVI  = (S1-S2)^2 (1-St*) [St*(S1+S2) + S1 S2 (1+St*)]
        //          / [(S1+S2)(St*+S1)(1+S1)(St*+S2)(1+S2)]
        //   dVII = (St*-d) sum_{s=S1,S2} [s (St*+d) + St* d] / [(s+St*)(s+d)]
        const float A = S1 + S2, P1 = S1 + Ss, P2 = S2 + Ss;
        const float Q1 = 1.0f + S1, Q2 = 1.0f + S2, R1 = S1 + d, R2 = S2 + d;
        const float dS = S1 - S2;
        const float nI = dS * dS * omSs * (Ss * A + S1 * S2 * (1.0f + Ss));
        const float dI = A * (P1 * Q1) * (P2 * Q2);
        const float sd = Ss + d, Sd = Ss * d;
        const float nII = Ssmd * ((S1 * sd + Sd) * (P2 * R2) + (S2 * sd + Sd) * (P1 * R1));
        const float dII = (P1 * R1) * (P2 * R2);
        const float V = fmaxf(nI / dI + nII / dII, 0.0f);
        const float vbm2 = pr[P3_U * N + i] + pr[P3_U * N + j];
        float dR, dP, dZ;
        if (has_vdust) {
            // input velocities: difference of FP32 hi/lo pairs
            dR = (pr[P3_VRH * N + i] - pr[P3_VRH * N + j]) + (pr[P3_VRL * N + i] - pr[P3_VRL * N + j]);
            dP = (pr[P3_VPH * N + i] - pr[P3_VPH * N + j]) + (pr[P3_VPL * N + i] - pr[P3_VPL * N + j]);
            dZ = (pr[P3_VZH * N + i] - pr[P3_VZH * N + j]) + (pr[P3_VZL * N + i] - pr[P3_VZL * N + j]);
        } else {
            // terminal velocities: differences factored through St_i - St_j
            //   v_R   = -2 eta v_K St/(1+St^2), v_phi = -eta v_K/(1+St^2),
            //   v_Z   = -Z Omega St/(1+St)
            const float dS = Si - Sj;
            const float ai = 1.0f + Si * Si, aj = 1.0f + Sj * Sj;
            const float rij = 1.0f / (ai * aj);
            const float ev = s4.z;
            dR = -2.0f * ev * dS * (1.0f - Si * Sj) * rij;
            dP = ev * dS * (Si + Sj) * rij;
            dZ = -s4.w * dS / ((1.0f + Si) * (1.0f + Sj));
        }
        const float dv2 = vbm2 + Vg2 * V + (dR * dR + dP * dP + dZ * dZ);
        const float dv = sqrtf(dv2);
        float K;
        if (kernel_mode == CUDISC_KERNEL_CONSTANT) K = kc;
        else if (kernel_mode == CUDISC_KERNEL_ADDITIVE) K = kc * (pr[P3_M * N + i] + pr[P3_M * N + j]);
        else { const float sa = pr[P3_A * N + i] + pr[P3_A * N + j]; K = 3.14159265358979f * sa * sa * dv; }
        float pf;
        if (frag_mode == CUDISC_FRAG_NONE) pf = 0.0f;
        else if (frag_mode == CUDISC_FRAG_ALL) pf = 1.0f;
        else {
            const float x = 1.5f * v_frag * v_frag / dv2;
            pf = (x + 1.0f) * expf(-x);
        }
        out = make_float2(K, K * pf);
    }
    Kout[(size_t)c * n_slots + q] = out;
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
        float2 v = K32[(size_t)c * n_slots + q];
        k = v.x; kf = v.y;
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
        for (int c0 = 0; c0 < c->n_cells; c0 += kMaxGridY) {
        dim3 grid((n_slots + 255) / 256, std::min(kMaxGridY, c->n_cells - c0));
        kbuild32_kernel<<<grid, 256, 0, c->stream>>>(
            c0, (float)p.kernel_const, (float)p.v_frag, p.kernel_mode, p.frag_mode, p.v_dust != nullptr,
            c->n_cells, c->N,
            n_slots, c->d_blk_i, c->d_blk_j0, c->d_a, c->d_minv, c->d_m, c->d_prep32, c->d_scal32,
            c->d_K32);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_get_kernel(const cudisc_coag_ctx *c, double *K, double *KF)
{
    for (int c0 = 0; c0 < c->n_cells; c0 += kMaxGridY) {
    dim3 grid((c->Np + 255) / 256, std::min(kMaxGridY, c->n_cells - c0));
    get_kernel_kernel<<<grid, 256, 0, c->stream>>>(c0, c->n_cells, c->Np, c->p.precision,
                                                   c->n_blk * kBlkPairs, c->d_pair_ij, c->d_K64,
                                                   c->d_K32, K, KF);
    }
    return cudaGetLastError();
}

} // namespace cdc
