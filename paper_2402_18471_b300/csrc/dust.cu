// Two pieces of the dust dynamics step of Sec. 3.1, data-parallel over
// cells x species: the source update of the full step (its items ii-iv and
// vi-viii) and the CFL time step (Eqs. dtCFL, dt_adv, dt_diff).
//
// Layout: conserved Q and primitive P fields [4][n_species][n_cells],
// Q = (rho, rho v_R, rho v_phi R, rho v_Z), P = (rho, v_R, v_phi, v_Z); gas
// fields per cell; v_g [3][n_cells].  A thread takes one cell and up to 8
// species (consecutive threads read consecutive cells of one species; the
// grid's second dimension covers the other species), so that the per-cell
// quantities are formed once per 8 species: Omega^2, 1/R and
// 1/(rho_g v_th).  FP64 throughout.
#include <cmath>

#include "coag_internal.h"

namespace cdc {
namespace {

constexpr int kDustThreads = 256;
constexpr int kSpecPerThread = 8;   // species a thread takes (grid.y covers the rest)

__global__ void __launch_bounds__(kDustThreads) dust_source_kernel(
    int n_s, int n_c, double *__restrict__ Q, const double *__restrict__ Pn, double h,
    const double *__restrict__ R, const double *__restrict__ Z, const double *__restrict__ rho_g,
    const double *__restrict__ c_s, const double *__restrict__ v_g, const double *__restrict__ a,
    double rho_m, double GM)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_c) return;
    const int s0 = blockIdx.y * kSpecPerThread;
    const int s1 = min(n_s, s0 + kSpecPerThread);
    const double Rc = R[c], Zc = Z[c];
    const double r2 = Rc * Rc + Zc * Zc;
    const double Om2 = GM / (r2 * sqrt(r2));                  // G M / (R^2 + Z^2)^(3/2)
    const double inv_R = 1.0 / Rc;
    const double vth = sqrt(8.0 / M_PI) * c_s[c];
    const double ts_per_a = rho_m / (rho_g[c] * vth);         // Epstein t_s = rho_m a / (rho_g v_th)
    const double vgR = v_g[c], vgP = v_g[(size_t)n_c + c], vgZ = v_g[2 * (size_t)n_c + c];
    const size_t plane = (size_t)n_s * n_c;
    for (int s = s0; s < s1; s++) {
        const size_t e = (size_t)s * n_c + c;
        const double rho_n = Pn[e], vphi_n = Pn[2 * plane + e];
        // explicit sources on the start-of-step primitives
        const double q0 = Q[e];
        const double q1 = Q[plane + e] + h * (rho_n * vphi_n * vphi_n * inv_R - rho_n * Om2 * Rc);
        const double q2 = Q[2 * plane + e];
        const double q3 = Q[3 * plane + e] + h * (-rho_n * Om2 * Zc);
        // primitives, then the implicit drag v <- v - h / (h + t_s) (v - v_g)
        const double inv_q0 = 1.0 / q0;
        double vR = q1 * inv_q0, vP = q2 * inv_q0 * inv_R, vZ = q3 * inv_q0;
        const double f = h / (h + ts_per_a * a[s]);
        vR -= f * (vR - vgR);
        vP -= f * (vP - vgP);
        vZ -= f * (vZ - vgZ);
        Q[plane + e] = q0 * vR;
        Q[2 * plane + e] = q0 * vP * Rc;
        Q[3 * plane + e] = q0 * vZ;
    }
}

// w[0] = dt, w[1] = the largest |v_R| / dR or |v_Z| / dZ (0: none), w[2] =
// the smallest Sc min(dR^2, dZ^2) / nu.  Both are positive doubles, whose
// bit patterns order as unsigned integers.
__global__ void dust_cfl_init(double *w)
{
    w[0] = INFINITY;
    w[1] = 0.0;
    w[2] = INFINITY;
}

// Per element only multiplications: the per-cell 1/dR, 1/dZ and
// min(dR^2, dZ^2) / nu are formed once per thread.  An input outside the
// domain of Eqs. dt_adv and dt_diff (a non-finite velocity; Sc, dR or dZ not
// positive and finite; nu negative or NaN) would otherwise drop out of the
// fmax/fmin reduction (or, negative, out of the unsigned atomicMin) and leave
// a plausible finite step: it sets w[1] to NaN instead, and so the result.
__global__ void __launch_bounds__(kDustThreads) dust_cfl_kernel(
    int n_s, int n_c, const double *__restrict__ P, const double *__restrict__ dR,
    const double *__restrict__ dZ, const double *__restrict__ nu, const double *__restrict__ Sc, double *w)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    double rate = 0.0, dif = INFINITY;
    bool bad = false;
    if (c < n_c) {
        const double dr = dR[c], dz = dZ[c], nc = nu[c];
        bad = !(fabs(dr) > 0.0) || !(fabs(dz) > 0.0) || !isfinite(dr) || !isfinite(dz) || !(nc >= 0.0);
        const double ir = 1.0 / fabs(dr), iz = 1.0 / fabs(dz);
        const double g = fmin(dr * dr, dz * dz) / nc;
        const size_t plane = (size_t)n_s * n_c;
        const int s0 = blockIdx.y * kSpecPerThread;
        const int s1 = min(n_s, s0 + kSpecPerThread);
        for (int s = s0; s < s1; s++) {
            const size_t e = (size_t)s * n_c + c;
            const double vr = P[plane + e], vz = P[3 * plane + e], sc = Sc[s];
            bad = bad || !isfinite(vr) || !isfinite(vz) || !(sc > 0.0) || !isfinite(sc);
            rate = fmax(rate, fmax(fabs(vr) * ir, fabs(vz) * iz));
            dif = fmin(dif, sc * g);
        }
    }
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
        dif = fmin(dif, __shfl_xor_sync(0xffffffffu, dif, o));
    }
    __shared__ double wr[kDustThreads / 32], wd[kDustThreads / 32];
    __shared__ int wb[kDustThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        wr[threadIdx.x >> 5] = rate;
        wd[threadIdx.x >> 5] = dif;
        wb[threadIdx.x >> 5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kDustThreads / 32; k++) {
            rate = fmax(rate, wr[k]);
            dif = fmin(dif, wd[k]);
            bad = bad || wb[k];
        }
        // a positive quiet NaN orders above every positive double as an
        // unsigned integer, so it survives the maximum
        if (bad) rate = __longlong_as_double(0x7FF8000000000000LL);
        if (bad || rate > 0.0)
            atomicMax(reinterpret_cast<unsigned long long *>(w + 1), (unsigned long long)__double_as_longlong(rate));
        if (dif < INFINITY)
            atomicMin(reinterpret_cast<unsigned long long *>(w + 2), (unsigned long long)__double_as_longlong(dif));
    }
}

__global__ void dust_cfl_finish(double *w, double C_adv, double C_diff)
{
    if (isnan(w[1])) { w[0] = w[1]; return; }
    const double adv = w[1] > 0.0 ? C_adv / w[1] : INFINITY;
    w[0] = fmin(adv, C_diff * w[2]);
}

} // namespace

cudaError_t launch_dust_source(int n_s, int n_c, double *Q, const double *Pn, double h, const double *R,
                               const double *Z, const double *rho_g, const double *c_s, const double *v_g,
                               const double *a, double rho_m, double GM, cudaStream_t stream)
{
    const dim3 grid((unsigned)((n_c + kDustThreads - 1) / kDustThreads),
                    (unsigned)((n_s + kSpecPerThread - 1) / kSpecPerThread));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    dust_source_kernel<<<grid, kDustThreads, 0, stream>>>(n_s, n_c, Q, Pn, h, R, Z, rho_g, c_s, v_g, a, rho_m, GM);
    return cudaGetLastError();
}

cudaError_t launch_dust_cfl(int n_s, int n_c, const double *P, const double *dR, const double *dZ,
                            const double *nu, const double *Sc, double C_adv, double C_diff, double *w,
                            cudaStream_t stream)
{
    const dim3 grid((unsigned)((n_c + kDustThreads - 1) / kDustThreads),
                    (unsigned)((n_s + kSpecPerThread - 1) / kSpecPerThread));
    if (grid.y > 65535) return cudaErrorInvalidValue;
    dust_cfl_init<<<1, 1, 0, stream>>>(w);
    dust_cfl_kernel<<<grid, kDustThreads, 0, stream>>>(n_s, n_c, P, dR, dZ, nu, Sc, w);
    dust_cfl_finish<<<1, 1, 0, stream>>>(w, C_adv, C_diff);
    return cudaGetLastError();
}

} // namespace cdc
