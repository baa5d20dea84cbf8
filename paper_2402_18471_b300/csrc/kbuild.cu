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
// terminal velocity at Z = h.  A block's threads share one cell: its
// scalars (sound speed, Omega, Re, ...; FP64 square roots and divisions)
// are formed once by the first thread.  The per-bin expressions keep the
// oracle's order of operations: the FP64 kernel's Ormel & Cuzzi terms and
// velocity differences amplify a one-ulp change of St or of a velocity where
// they cancel.
__global__ void __launch_bounds__(128) prep_kernel(
    int c0, KParams kp, int n_cells, int N, const double *__restrict__ a, const double *__restrict__ minv,
    const double *__restrict__ m, const double *__restrict__ rho_gas, const double *__restrict__ T,
    const double *__restrict__ alpha, const double *__restrict__ R,
    const double *__restrict__ Z, const double *__restrict__ eta,
    const double *__restrict__ v_dust, double *__restrict__ prep,
    float *__restrict__ prep32, CellScal *__restrict__ scal, float4 *__restrict__ scal32)
{
    const int c = c0 + blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;                 // uniform over the block
    // per-cell scalars: d, rho_g v_th, 8 k_B T / pi, eta v_K, Z (or 0), Omega, H, alpha, v_K
    __shared__ double sc[9];
    if (threadIdx.x == 0) {
        const double Tc = T[c], rg = rho_gas[c], Rc = R[c], Zc = kp.vertical ? 0.0 : Z[c], al = alpha[c];
        const double cs = sqrt(kp.k_B * Tc / (kp.mu * kp.m_H));
        const double vth = sqrt(8.0 / M_PI) * cs;
        const double r2 = Rc * Rc + Zc * Zc;
        const double Om = sqrt(kp.G * kp.Mstar / (r2 * sqrt(r2)));
        const double Om_mid = sqrt(kp.G * kp.Mstar / (Rc * Rc * Rc));
        const double nu_t = al * cs * (cs / Om_mid);
        const double nu_mol = 0.5 * vth * (kp.mu * kp.m_H / (rg * kp.sigma_H2));
        const double delta = 1.0 / sqrt(nu_t / nu_mol);
        const double etavK = (eta ? eta[c] : 0.0) * Om * Rc;
        sc[0] = delta;
        sc[1] = rg * vth;
        sc[2] = 8.0 * kp.k_B * Tc / M_PI;
        sc[3] = etavK;
        sc[4] = Zc;
        sc[5] = Om;
        sc[6] = cs / Om_mid;
        sc[7] = al;
        sc[8] = Om * Rc;
        if (blockIdx.x == 0) {
            CellScal s;
            s.kT8pi = sc[2];
            s.Vg2 = al * cs * cs;
            s.delta = delta;
            s.etavK = etavK;
            s.ZOm = Zc * Om;
            s.pad = 0.0;
            scal[c] = s;
            scal32[c] = make_float4((float)s.delta, (float)s.Vg2, (float)s.etavK, (float)s.ZOm);
        }
    }
    __syncthreads();
    if (k >= N) return;
    const double delta = sc[0], Om = sc[5], al = sc[7];
    const double St = kp.rho_m * a[k] / sc[1] * Om;
    const double hk = kp.vertical ? sc[6] * sqrt(al / (al + St)) : 0.0;
    double vR, vphi, vZ;
    if (v_dust) {
        const size_t nc = (size_t)n_cells * N;
        vR = v_dust[(size_t)c * N + k];
        vphi = v_dust[nc + (size_t)c * N + k];
        vZ = v_dust[2 * nc + (size_t)c * N + k];
    } else {
        const double et = eta ? eta[c] : 0.0, vK = sc[8];
        vR = -2.0 * et * vK * St / (1.0 + St * St);
        vphi = -et * vK / (1.0 + St * St);
        vZ = -(kp.vertical ? hk : sc[4]) * Om * St / (1.0 + St);
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
                                 (float)(1.0 - Ss), (float)(sc[2] * minv[k]),
                                 (float)a[k], (float)m[k], (float)(2.0 * M_PI * hk * hk)};
#pragma unroll
    for (int f = 0; f < P3_COUNT; f++) pf[f * N + k] = v32[f];
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

// One 32-byte global store (a whole sector: the four slots of a thread go
// out in one piece, so that a warp's 1 KB is 32 full sectors; two 16-byte
// stores at a 32-byte lane stride would each fill half of 32 sectors).  p
// must be 32-byte aligned.
__device__ __forceinline__ void st_global_v8(void *p, const float (&o)[8])
{
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3]), "f"(o[4]), "f"(o[5]), "f"(o[6]), "f"(o[7])
                 : "memory");
}

// Packed FP32 pairs: two lanes in one 64-bit register, one instruction for
// both (add/sub/mul/fma .rn .f32x2: the same IEEE round-to-nearest as two
// scalar ones), which halves the FP32 issue of the builder's pair loop.
struct F2 { unsigned long long r; };
__device__ __forceinline__ F2 f2(float a, float b)
{
    F2 o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(a), "f"(b));
    return o;
}
__device__ __forceinline__ void f2s(F2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v.r));
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 o;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 o;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    F2 o;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c)
{
    F2 o;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(o.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return o;
}
__device__ __forceinline__ F2 rcp2(F2 v)
{
    float a, b;
    f2s(v, a, b);
    return f2(rcp_ftz(a), rcp_ftz(b));
}
__device__ __forceinline__ F2 rsqrt2(F2 v)
{
    float a, b;
    f2s(v, a, b);
    return f2(rsqrt_ftz(a), rsqrt_ftz(b));
}
// 2^v per lane
__device__ __forceinline__ F2 ex2_2(F2 v)
{
    float a, b, ra, rb;
    f2s(v, a, b);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ra) : "f"(a));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(rb) : "f"(b));
    return f2(ra, rb);
}

// Coagulation probability p_c = 1 - (1 + x) e^-x of Eq. (p_frag), accurate in
// FP32 also where p_frag rounds to 1: for x < 1 as x^2 g(x) with
//   g(x) = (1 - (1 + x) e^-x) / x^2 = e^-x sum_{m>=0} x^m / (m + 2)!,
// a smooth function with g(0) = 1/2, approximated on [0, 1] by its degree-6
// Chebyshev interpolant (interpolation error 6e-9 relative; evaluated by
// Horner in FP32 it is as accurate as the 13-term Taylor series it replaces,
// 1.6e-7); for x >= 1 from the closed form (p_c >= 0.26 there, no
// cancellation) as 1 - p_frag.  Given p_frag = (1 + x) e^-x.  The
// coefficients are computed on the host (pcoag_poly).
struct PcoagPoly { float c[7]; };   // monomial coefficients, c[0] the constant term

__device__ __forceinline__ float pcoag_f32(float x, float pf, const PcoagPoly &P)
{
    if (x >= 1.0f) return 1.0f - pf;
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
// 16, zero-padded so that four consecutive bins load as one 16-byte word).
// For bin k of a cell, with S = St_k, S* = St*_k (the clamp it takes when it
// is the larger of a pair), d = Re^-1/2 and V_g^2 = alpha c_s^2:
//   KB_S   S                      KB_U   8 k_B T / (pi m_k)
//   KB_SS  S*                     KB_SA  sqrt(pi) a_k
//   KB_OPSS 1 + S*                KB_IQ  1 / (1 + S)
//   KB_W1  V_g^2 (1 - S*) / ((S* + S)(1 + S))
//   KB_KD1 V_g^2 (S* - d)(S* + d) KB_IR  1 / (S + d)
//   KB_KD0 V_g^2 (S* - d) S* d
//   KB_EV  V_g^2 (S* - d) [S (S* + d) + S* d] / ((S + S*)(S + d))
// and then either, for the terminal velocities,
//   KB_EA  (eta v_K / (1 + S^2))^2  KB_ZQ  (Z Omega / (1 + S))^2
//   KB_IA2 1 / (1 + S^2)^2          KB_IQ2 1 / (1 + S)^2
// or, for input velocities and the vertically integrated kernel, the prep
// kernel's FP32 hi/lo velocity pairs in the same places (KB_VRH .. KB_VZL);
// last KB_HH = 2 pi h^2 (vertically integrated kernel) and KB_M = m_k (the
// closed-form test kernels).  Everything a pair needs from one of its bins
// is thus formed once per bin, in FP32 from the prep kernel's values (the
// differences S* - d and 1 - S* come from FP64 there).
enum {
    KB_S = 0, KB_SS, KB_OPSS, KB_W1, KB_KD1, KB_KD0, KB_EV, KB_U, KB_SA, KB_IQ, KB_IR,
    KB_EA, KB_ZQ, KB_IA2, KB_IQ2, KB_HH = KB_EA + 6, KB_M, KB_COUNT
};
enum { KB_VRH = KB_EA, KB_VRL, KB_VPH, KB_VPL, KB_VZH, KB_VZL };

// The per-bin fields above (terminal-velocity ones included) of a bin with
// prep values St, St*, St* - d, 1 - St*, U and a in a cell with scalars
// s4 = {d, V_g^2, eta v_K, Z Omega}.
struct BinF { float S, Ss, opSs, W1, KD1, KD0, EV, U, SA, IQ, IR, EA, ZQ, IA2, IQ2; };
__device__ __forceinline__ BinF bin_fields_from(float S, float Ss, float Ssmd, float omSs, float U, float a,
                                                float4 s4)
{
    BinF v;
    const float d = s4.x, Vg2 = s4.y;
    const float sd = Ss + d, Sd = Ss * d, vs = Vg2 * Ssmd;
    v.S = S;
    v.Ss = Ss;
    v.opSs = 1.0f + Ss;
    v.W1 = Vg2 * omSs * rcp_ftz((Ss + S) * (1.0f + S));
    v.KD1 = vs * sd;
    v.KD0 = vs * Sd;
    v.EV = vs * (S * sd + Sd) * rcp_ftz((S + Ss) * (S + d));
    v.U = U;
    v.SA = 1.7724538509055160f * a;
    v.IQ = rcp_ftz(1.0f + S);
    v.IR = rcp_ftz(S + d);
    const float ia = rcp_ftz(1.0f + S * S);
    const float ea = s4.z * ia, zq = s4.w * v.IQ;
    v.EA = ea * ea;
    v.ZQ = zq * zq;
    v.IA2 = ia * ia;
    v.IQ2 = v.IQ * v.IQ;
    return v;
}
// the same from the prep kernel's fields of the bin at P (stride N)
__device__ __forceinline__ BinF bin_fields(const float *__restrict__ P, int N, float4 s4)
{
    return bin_fields_from(P[P3_ST * N], P[P3_SS * N], P[P3_SSMD * N], P[P3_OMSS * N], P[P3_U * N], P[P3_A * N], s4);
}

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
// fields (above) are formed in shared memory once; each thread then produces
// four consecutive slots of a block (same i, j .. j+3) and writes them as two
// 16-byte chunks, a warp 1 KB of its cell's table per store pair.  The
// larger Stokes number of a pair (i, j <= i) is always St_i: St = rho_m a
// Omega / (rho_g v_th) rises with the bin's size.
//
// Per pair, with S1 = St_i >= S2 = St_j, A = S1 + S2, dS = S1 - S2 and
// B = S* A + S1 S2 (1 + S*) (S*, d of bin i), the Ormel & Cuzzi class I and
// II terms are, algebraically identical to the closed forms,
//   V_g^2 dVI  = dS^2 / A * W1_i * B * IQ_j / (S* + S2)
//   V_g^2 dVII = EV_i + (KD1_i S2 + KD0_i) * IR_j / (S* + S2)
// (class II summed per particle: (S* - d) + s^2/(s + S*) - s^2/(s + d) =
// (S* - d)[s (S* + d) + S* d] / ((s + S*)(s + d))), and the terminal
// velocities' differences factor through dS:
//   dv_lam^2 = dS^2 [EA_i IA2_j (4 (1 - S1 S2)^2 + A^2) + ZQ_i IQ2_j].
// Every factor is non-negative, so nothing cancels in FP32 (the literal
// forms do: with S* clamped to d and S1 = S2 class II is exactly zero but
// leaves a residue ~1e-7 S^2/d, and for St >> 1 both reduce to small
// differences of numbers near one), and a pair costs two reciprocals, a
// reciprocal square root and an exponential besides ~40 FP32 operations.
// Those use the hardware approximations: K stays within 1e-6 and K p_frag
// within 1e-5 of FP64.
//   Physical = physical kernel and fragmentation probability (the other
//   modes are the closed-form test kernels); HasVdust = input velocities.
constexpr int kWarpsPerCell = 4;            // warps sharing one cell's table
constexpr int kPosTile = 8 / kWarpsPerCell; // cells per CTA of 256 threads

// words of shared memory per cell
__host__ __device__ inline int kb_cell_stride(int NR) { return KB_COUNT * NR; }

template <bool Physical, bool HasVdust>
__global__ void __launch_bounds__(256) kbuild32_kernel(
    float kc, float v_frag, int kernel_mode, int frag_mode, int vertical, int n_cells, int N, int NR,
    int n_slots, const int *__restrict__ blk_i, const int *__restrict__ blk_j0,
    const float *__restrict__ prep32, const float4 *__restrict__ scal32, PcoagPoly poly,
    float2 *__restrict__ Kout)
{
    extern __shared__ __align__(16) float f32s[];       // [kPosTile][KB_COUNT][NR]
    const int CS = kb_cell_stride(NR);
    const int cell0 = blockIdx.x * kPosTile;
    __shared__ int s_cell[kPosTile];
    if (threadIdx.x < kPosTile) {
        const int c = cell0 + (int)threadIdx.x;
        s_cell[threadIdx.x] = c < n_cells ? c : -1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kPosTile * NR; t += blockDim.x) {
        const int jc = t / NR, k = t - jc * NR;
        const int c = s_cell[jc];
        float *F = f32s + jc * CS + k;
        if (c < 0 || k >= N) {
            for (int f = 0; f < KB_COUNT; f++) F[f * NR] = 0.0f;
            continue;
        }
        const float *P = prep32 + (size_t)c * P3_COUNT * N + k;
        const BinF v = bin_fields(P, N, scal32[c]);
        F[KB_S * NR] = v.S;
        F[KB_SS * NR] = v.Ss;
        F[KB_OPSS * NR] = v.opSs;
        F[KB_W1 * NR] = v.W1;
        F[KB_KD1 * NR] = v.KD1;
        F[KB_KD0 * NR] = v.KD0;
        F[KB_EV * NR] = v.EV;
        F[KB_U * NR] = v.U;
        F[KB_SA * NR] = v.SA;
        F[KB_IQ * NR] = v.IQ;
        F[KB_IR * NR] = v.IR;
        if (!HasVdust) {
            F[KB_EA * NR] = v.EA;
            F[KB_ZQ * NR] = v.ZQ;
            F[KB_IA2 * NR] = v.IA2;
            F[KB_IQ2 * NR] = v.IQ2;
        } else {
            F[KB_VRH * NR] = P[P3_VRH * N];
            F[KB_VRL * NR] = P[P3_VRL * N];
            F[KB_VPH * NR] = P[P3_VPH * N];
            F[KB_VPL * NR] = P[P3_VPL * N];
            F[KB_VZH * NR] = P[P3_VZH * N];
            F[KB_VZL * NR] = P[P3_VZL * N];
        }
        F[KB_HH * NR] = vertical ? P[P3_HH * N] : 0.0f;
        F[KB_M * NR] = Physical ? 0.0f : P[P3_M * N];
    }
    __syncthreads();
    const int jc = (threadIdx.x >> 5) / kWarpsPerCell;    // this warp's cell of the tile
    const int part = (threadIdx.x >> 5) % kWarpsPerCell;  // and its share of the cell's groups
    const int c = s_cell[jc];
    if (c < 0) return;
    const float *F = f32s + jc * CS;
    const float vf2 = 1.5f * v_frag * v_frag;
    float4 *dst = reinterpret_cast<float4 *>(Kout) + (size_t)c * (n_slots / 2);   // the cell's 2-pair chunks
    const int n_grp = n_slots / 4;
    const int g_end = (int)((long long)(part + 1) * n_grp / kWarpsPerCell);
    auto f4 = [&](int f, int j) { return *reinterpret_cast<const float4 *>(F + f * NR + j); };
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
        float o[8];
        {
        // bin i (the larger Stokes number)
        const float S1 = F[KB_S * NR + i], Ss = F[KB_SS * NR + i], opSs = F[KB_OPSS * NR + i];
        const float W1 = F[KB_W1 * NR + i], KD1 = F[KB_KD1 * NR + i], KD0 = F[KB_KD0 * NR + i];
        const float EV = F[KB_EV * NR + i], Ui = F[KB_U * NR + i], SAi = F[KB_SA * NR + i];
        // bins j0 .. j0+3
        const float4 v_S = f4(KB_S, j0), v_U = f4(KB_U, j0), v_SA = f4(KB_SA, j0);
        const float4 v_IQ = f4(KB_IQ, j0), v_IR = f4(KB_IR, j0);
        const float S2a[4] = {v_S.x, v_S.y, v_S.z, v_S.w};
        const float Uja[4] = {v_U.x, v_U.y, v_U.z, v_U.w};
        const float SAa[4] = {v_SA.x, v_SA.y, v_SA.z, v_SA.w};
        const float IQa[4] = {v_IQ.x, v_IQ.y, v_IQ.z, v_IQ.w};
        const float IRa[4] = {v_IR.x, v_IR.y, v_IR.z, v_IR.w};
        float EAi = 0.f, ZQi = 0.f, IA2a[4] = {}, IQ2a[4] = {};
        if (!HasVdust) {
            EAi = F[KB_EA * NR + i];
            ZQi = F[KB_ZQ * NR + i];
            const float4 v_IA2 = f4(KB_IA2, j0), v_IQ2 = f4(KB_IQ2, j0);
            IA2a[0] = v_IA2.x; IA2a[1] = v_IA2.y; IA2a[2] = v_IA2.z; IA2a[3] = v_IA2.w;
            IQ2a[0] = v_IQ2.x; IQ2a[1] = v_IQ2.y; IQ2a[2] = v_IQ2.z; IQ2a[3] = v_IQ2.w;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int j = j0 + u;
            const float S2 = S2a[u];
            const float A = S1 + S2, dS = S1 - S2, S12 = S1 * S2;
            const float rA = rcp_ftz(A), rP = rcp_ftz(Ss + S2);
            const float dS2 = dS * dS;
            const float B = fmaf(S12, opSs, Ss * A);
            const float tI = (dS2 * rA) * B * (W1 * IQa[u]);
            const float tII = fmaf(S2, KD1, KD0) * IRa[u];
            const float vt = fmaf(tI + tII, rP, EV);        // V_g^2 (dVI + dVII)
            float lam;
            if (!HasVdust) {
                const float w2 = fmaf(S12, -2.0f, 2.0f);
                const float Lr = fmaf(w2, w2, A * A);
                lam = dS2 * fmaf(EAi * IA2a[u], Lr, ZQi * IQ2a[u]);
            } else {
                // input velocities: difference of FP32 hi/lo pairs
                const float dR = (F[KB_VRH * NR + i] - F[KB_VRH * NR + j]) + (F[KB_VRL * NR + i] - F[KB_VRL * NR + j]);
                const float dP = (F[KB_VPH * NR + i] - F[KB_VPH * NR + j]) + (F[KB_VPL * NR + i] - F[KB_VPL * NR + j]);
                const float dZ = (F[KB_VZH * NR + i] - F[KB_VZH * NR + j]) + (F[KB_VZL * NR + i] - F[KB_VZL * NR + j]);
                lam = fmaf(dR, dR, fmaf(dP, dP, dZ * dZ));
            }
            const float dv2 = lam + (vt + (Ui + Uja[u]));
            const float rs = rsqrt_ftz(dv2);
            float K, pc, pf;
            if (Physical) {
                const float sa = SAi + SAa[u];
                K = sa * sa * (dv2 * rs);
                const float x = vf2 * (rs * rs);
                const float e = exp_neg_ftz(x);
                pf = fmaf(x, e, e);
                pc = pcoag_f32(x, pf, poly);
            } else {
                if (kernel_mode == CUDISC_KERNEL_CONSTANT) K = kc;
                else if (kernel_mode == CUDISC_KERNEL_ADDITIVE) K = kc * (F[KB_M * NR + i] + F[KB_M * NR + j]);
                else { const float sa = SAi + SAa[u]; K = sa * sa * (dv2 * rs); }
                if (frag_mode == CUDISC_FRAG_NONE) { pf = 0.0f; pc = 1.0f; }
                else if (frag_mode == CUDISC_FRAG_ALL) { pf = 1.0f; pc = 0.0f; }
                else {
                    const float x = vf2 * (rs * rs);
                    const float e = exp_neg_ftz(x);
                    pf = fmaf(x, e, e);
                    pc = pcoag_f32(x, pf, poly);
                }
            }
            if (vertical) K *= rsqrt_ftz(F[KB_HH * NR + i] + F[KB_HH * NR + j]);
            o[2 * u] = K * pc;
            o[2 * u + 1] = K * pf;
        }
        }
        if (j0 + 3 > i) {
            // the block's diagonal group: zero the slots past it
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (j0 + u > i) o[2 * u] = o[2 * u + 1] = 0.0f;
        }
        dst[2 * g] = make_float4(o[0], o[1], o[2], o[3]);
        dst[2 * g + 1] = make_float4(o[4], o[5], o[6], o[7]);
    }
}

// The physical kernel with terminal velocities (the paper's case and the
// common one) in packed FP32 lanes: two slots per instruction, the same
// arithmetic as kbuild32_kernel.  Per cell, shared memory holds for every
// bin the fields a pair takes from its larger bin as duplicated pairs
// {v, v} (one 96-byte record, KD_*, read by all lanes of a block row at
// once) and the fields a pair takes from its smaller bin field-major with a
// fixed stride of kMaxNR (KJ_*: neighbouring lanes read neighbouring 16-byte
// words, conflict-free), so that a thread's four slots load their operands
// as thirteen 16-byte words at fixed offsets; the block table is staged as
// i << 16 | j0 per 16-pair block.
enum { KD_S = 0, KD_SS, KD_OPSS, KD_W1, KD_KD1, KD_KD0, KD_EV, KD_U, KD_SA, KD_EA, KD_ZQ, KD_STRIDE = 12 };
enum { KJ_S = 0, KJ_IQ, KJ_IR, KJ_IA2, KJ_IQ2, KJ_U, KJ_SA, KJ_COUNT };
constexpr int kMaxNR = (kMaxBins + 15) / 16 * 16;   // the largest padded bin count
__host__ __device__ inline int kbf_cell_floats(int NR) { return 2 * KD_STRIDE * NR + KJ_COUNT * kMaxNR; }
constexpr int kFastThreads = 128;           // one cell per CTA, four warps

// One CTA per cell: the cell's derived fields and the block table are
// formed in shared memory, then the four warps take interleaved runs of 32
// groups of the cell, so that together they write its table front to back.
// (A persistent variant that fetched the next cell's prep values while
// writing one measured 10 % slower than these independent CTAs, eight of
// which an SM holds.)
__global__ void __launch_bounds__(kFastThreads, 1024 / kFastThreads) kbuild32_fast_kernel(
    float v_frag, int n_cells, int N, int NR, int n_slots, int n_blk, const int *__restrict__ blk_i,
    const int *__restrict__ blk_j0, const float *__restrict__ prep32, const float4 *__restrict__ scal32,
    PcoagPoly poly, float2 *__restrict__ Kout)
{
    extern __shared__ __align__(16) float f32s[];   // the cell's fields, then int [n_blk]
    const float *F = f32s;
    int *s_blk = reinterpret_cast<int *>(f32s + kbf_cell_floats(NR));
    const int c = blockIdx.x;
    if (c >= n_cells) return;
    for (int b = threadIdx.x; b < n_blk; b += blockDim.x) s_blk[b] = (__ldg(blk_i + b) << 16) | __ldg(blk_j0 + b);
    const float4 s4 = scal32[c];
    for (int k = threadIdx.x; k < NR; k += blockDim.x) {
        float vi[KD_STRIDE] = {}, vj[KJ_COUNT] = {};
        if (k < N) {
            const BinF v = bin_fields(prep32 + (size_t)c * P3_COUNT * N + k, N, s4);
            vi[KD_S] = v.S; vi[KD_SS] = v.Ss; vi[KD_OPSS] = v.opSs; vi[KD_W1] = v.W1;
            vi[KD_KD1] = v.KD1; vi[KD_KD0] = v.KD0; vi[KD_EV] = v.EV; vi[KD_U] = v.U;
            vi[KD_SA] = v.SA; vi[KD_EA] = v.EA; vi[KD_ZQ] = v.ZQ;
            vj[KJ_S] = v.S; vj[KJ_IQ] = v.IQ; vj[KJ_IR] = v.IR; vj[KJ_IA2] = v.IA2;
            vj[KJ_IQ2] = v.IQ2; vj[KJ_U] = v.U; vj[KJ_SA] = v.SA;
        }
        float2 *DI = reinterpret_cast<float2 *>(f32s) + k * KD_STRIDE;
        float *DJ = f32s + 2 * KD_STRIDE * NR + k;
#pragma unroll
        for (int f = 0; f < KD_STRIDE; f++) DI[f] = make_float2(vi[f], vi[f]);
#pragma unroll
        for (int f = 0; f < KJ_COUNT; f++) DJ[f * kMaxNR] = vj[f];
    }
    __syncthreads();
    const int part = threadIdx.x >> 5;                   // this warp's runs of the cell's groups
    const float vf2 = 1.5f * v_frag * v_frag;
    const F2 two = f2(2.0f, 2.0f), mtwo = f2(-2.0f, -2.0f), one = f2(1.0f, 1.0f);
    const F2 vf = f2(vf2, vf2), vfl = f2(-1.4426950408889634f * vf2, -1.4426950408889634f * vf2);
    F2 pcf[7];
#pragma unroll
    for (int k = 0; k < 7; k++) pcf[k] = f2(poly.c[k], poly.c[k]);
    const int n_grp = n_slots / 4;
    float4 *dst = reinterpret_cast<float4 *>(Kout) + (size_t)c * (n_slots / 2);   // the cell's 2-pair chunks
    for (int g = 32 * part + (threadIdx.x & 31); g < n_grp; g += kFastThreads) {
        const int q0 = 4 * g;
        const int bij = s_blk[q0 >> 4];
        const int i = bij >> 16;
        const int j0 = (bij & 0xffff) + (q0 & 15);
        if (j0 > i) continue;   // all four slots past the diagonal: zero since allocation
        // bin i (the larger Stokes number) in both lanes
        const ulonglong2 *RI = reinterpret_cast<const ulonglong2 *>(F) + i * (KD_STRIDE / 2);
        F2 di[KD_STRIDE];
#pragma unroll
        for (int w = 0; w < KD_STRIDE / 2; w++) {
            const ulonglong2 v = RI[w];
            di[2 * w].r = v.x;
            di[2 * w + 1].r = v.y;
        }
        // bins j0, j0+1 and j0+2, j0+3: the lanes of h = 0 and h = 1
        const float *RJ = F + 2 * KD_STRIDE * NR + j0;
        F2 dj[KJ_COUNT][2];
#pragma unroll
        for (int w = 0; w < KJ_COUNT; w++) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(RJ + w * kMaxNR);
            dj[w][0].r = v.x;
            dj[w][1].r = v.y;
        }
        const F2 S1 = di[KD_S], Ss = di[KD_SS];
        float o[8];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const F2 S2 = dj[KJ_S][h];
            const F2 A = S1 + S2, dS = S1 - S2, S12 = S1 * S2;
            // both classes over the common denominator A (S* + S2): one reciprocal
            const F2 r = rcp2(A * (Ss + S2));
            const F2 dS2 = dS * dS;
            const F2 B = fma2(S12, di[KD_OPSS], Ss * A);
            const F2 tI = (dS2 * B) * (di[KD_W1] * dj[KJ_IQ][h]);
            const F2 tII = fma2(S2, di[KD_KD1], di[KD_KD0]) * dj[KJ_IR][h];
            const F2 vt = fma2(fma2(tII, A, tI), r, di[KD_EV]);   // V_g^2 (dVI + dVII)
            const F2 w2 = fma2(S12, mtwo, two);
            const F2 Lr = fma2(w2, w2, A * A);
            const F2 lam = dS2 * fma2(di[KD_EA] * dj[KJ_IA2][h], Lr, di[KD_ZQ] * dj[KJ_IQ2][h]);
            const F2 dv2 = lam + (vt + (di[KD_U] + dj[KJ_U][h]));
            const F2 rs = rsqrt2(dv2);
            const F2 sa = di[KD_SA] + dj[KJ_SA][h];
            const F2 K = sa * sa * (dv2 * rs);
            const F2 rs2 = rs * rs;
            const F2 x = vf * rs2;
            const F2 e = ex2_2(vfl * rs2);                          // e^-x
            const F2 pf = fma2(x, e, e);
            F2 sp = pcf[6];
#pragma unroll
            for (int k = 5; k >= 0; k--) sp = fma2(sp, x, pcf[k]);
            const F2 pcs = (x * x) * sp, pcl = one - pf;           // p_c below and above x = 1
            float xa, xb, sa_, sb_, la, lb;
            f2s(x, xa, xb);
            f2s(pcs, sa_, sb_);
            f2s(pcl, la, lb);
            // the products as scalars, written in slot order for the store
            float Ka, Kb, pfa, pfb;
            f2s(K, Ka, Kb);
            f2s(pf, pfa, pfb);
            o[4 * h] = Ka * (xa >= 1.0f ? la : sa_);
            o[4 * h + 1] = Ka * pfa;
            o[4 * h + 2] = Kb * (xb >= 1.0f ? lb : sb_);
            o[4 * h + 3] = Kb * pfb;
        }
        if (j0 + 3 > i) {
            // the block's diagonal group: zero the slots past it
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (j0 + u > i) o[2 * u] = o[2 * u + 1] = 0.0f;
        }
        st_global_v8(dst + 2 * g, o);
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
    prep_kernel<<<grid, 128, 0, c->stream>>>(c0, kparams(p), c->n_cells, c->N, c->d_a, c->d_minv, c->d_m, p.rho_gas, p.T,
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
        const size_t smem = (size_t)kPosTile * kb_cell_stride(NR) * sizeof(float);
        const bool phys = p.kernel_mode == CUDISC_KERNEL_PHYSICAL && p.frag_mode == CUDISC_FRAG_PHYSICAL;
        // the vertically integrated kernel's settling velocities (each grain
        // at its own height) do not factor through St_i - St_j: take the
        // differences of the prep kernel's FP32 hi/lo velocity pairs
        const bool vd = p.v_dust != nullptr || p.vertical;
        static const PcoagPoly poly = pcoag_poly();
        if (phys && !vd) {
            const size_t fsmem = (size_t)kbf_cell_floats(NR) * sizeof(float) + (size_t)c->n_blk * sizeof(int);
            cudaError_t e = cudaFuncSetAttribute(kbuild32_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)fsmem);
            if (e != cudaSuccess) return e;
            kbuild32_fast_kernel<<<c->n_cells, kFastThreads, fsmem, c->stream>>>(
                (float)p.v_frag, c->n_cells, c->N, NR, n_slots, c->n_blk, c->d_blk_i, c->d_blk_j0, c->d_prep32,
                c->d_scal32, poly, c->d_K32);
            return cudaGetLastError();
        }
        auto kern = phys ? kbuild32_kernel<true, true> : (vd ? kbuild32_kernel<false, true> : kbuild32_kernel<false, false>);
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
