// Gas density from hydrostatic equilibrium (Sec. 3.5, Eqs. hydroeqbm,
// hedisc, avcs, heprod, rhonorm): per column of the (R, Z) grid, the ratio
// of each cell's pressure to the one below it,
//   P_j / P_{j-1} = exp[G M_* <1/c_s^2>_j (1/r_j - 1/r_{j-1})],
//   <1/c_s^2>_j = (1/c_s,j^2 + 1/c_s,j-1^2) / 2,
// their running product P_j / P_0 (a multiplicative scan, which keeps the
// pressure positive), the density P / c_s^2, and its normalisation to the
// column's surface density, rho_j = Sigma_g (R dR) / (sum_k omega_k V_k)
// omega_j.  The result is the gas density the collision-kernel builder
// reads.
//
// One warp per column: each pass over 32 consecutive cells (coalesced reads
// of T, R, Z and V) forms the ratios from the lane below (shuffles; the
// previous pass's last cell for lane 0), scans them with five shuffle
// multiplications, carries the product to the next pass, writes the
// unnormalised density and accumulates sum omega V; a second pass over the
// column (its writes are still in L2) applies the normalisation.  FP64
// throughout: the exponent is a difference of nearly equal 1/r.
#include "coag_internal.h"

namespace cdc {
namespace {

constexpr int kHseThreads = 256;   // 8 columns per block

// e^x for the per-cell exponents, which are small on any but the coarsest
// columns: for |x| <= 1/8 the Taylor series sum_{n<=12} x^n / n! by Horner
// (truncation below (1/8)^13 / 13! = 1e-21 relative), else exp().  B300's
// FP64 rate is a small fraction of its FP32 rate and this kernel is bound by
// it: 12 FMAs in place of the library's range reduction and polynomial.
__device__ __forceinline__ double exp_small(double x)
{
    if (fabs(x) > 0.125) return exp(x);
    double s = 1.0 / 479001600.0;                       // 1/12!
    s = fma(s, x, 1.0 / 39916800.0);
    s = fma(s, x, 1.0 / 3628800.0);
    s = fma(s, x, 1.0 / 362880.0);
    s = fma(s, x, 1.0 / 40320.0);
    s = fma(s, x, 1.0 / 5040.0);
    s = fma(s, x, 1.0 / 720.0);
    s = fma(s, x, 1.0 / 120.0);
    s = fma(s, x, 1.0 / 24.0);
    s = fma(s, x, 1.0 / 6.0);
    s = fma(s, x, 0.5);
    s = fma(s, x, 1.0);
    return fma(s, x, 1.0);
}

__global__ void __launch_bounds__(kHseThreads) hse_kernel(
    int n_R, int n_Z, const double *__restrict__ R, const double *__restrict__ Z,
    const double *__restrict__ T, const double *__restrict__ V, const double *__restrict__ R_edges,
    const double *__restrict__ Sigma_g, double mu_mH_over_kB, double GM, double *__restrict__ rho)
{
    const int col = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= n_R) return;                                // whole warps leave together
    const size_t base = (size_t)col * n_Z;
    const unsigned full = 0xffffffffu;
    double carry = 1.0;                                    // P_{j0-1} / P_0
    double ics2_prev = 0.0, ir_prev = 0.0;                 // 1/c_s^2 and 1/r of cell j0 - 1
    double wsum = 0.0;
    for (int j0 = 0; j0 < n_Z; j0 += 32) {
        const int j = j0 + lane;
        const bool in = j < n_Z;
        double ics2 = 0.0, ir = 0.0;
        if (in) {
            ics2 = mu_mH_over_kB / T[base + j];            // 1 / c_s^2 = mu m_H / (k_B T)
            const double rr = R[base + j], zz = Z[base + j];
            ir = rsqrt(fma(rr, rr, zz * zz));
        }
        double ics2_m = __shfl_up_sync(full, ics2, 1), ir_m = __shfl_up_sync(full, ir, 1);
        if (lane == 0) { ics2_m = ics2_prev; ir_m = ir_prev; }
        double q = 1.0;                                    // P_j / P_{j-1} (1 at j = 0 and past the column)
        if (in && j > 0) q = exp_small(GM * (0.5 * (ics2 + ics2_m)) * (ir - ir_m));
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(full, q, o);
            if (lane >= o) q *= v;
        }
        const double p = carry * q;                        // P_j / P_0
        if (in) {
            const double om = p * ics2;                    // unnormalised density P / c_s^2
            rho[base + j] = om;
            wsum += om * V[base + j];
        }
        carry = __shfl_sync(full, p, 31);
        ics2_prev = __shfl_sync(full, ics2, 31);
        ir_prev = __shfl_sync(full, ir, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(full, wsum, o);
    const double re0 = R_edges[col], re1 = R_edges[col + 1];
    const double s = Sigma_g[col] * (0.5 * (re1 * re1 - re0 * re0)) / wsum;
    __syncwarp();
    for (int j = lane; j < n_Z; j += 32) rho[base + j] *= s;
}

} // namespace

cudaError_t launch_hse(int n_R, int n_Z, const double *R, const double *Z, const double *T, const double *V,
                       const double *R_edges, const double *Sigma_g, double mu, double m_H, double k_B,
                       double GM, double *rho, cudaStream_t stream)
{
    const int per_block = kHseThreads / 32;
    const unsigned blocks = (unsigned)((n_R + per_block - 1) / per_block);
    hse_kernel<<<blocks, kHseThreads, 0, stream>>>(n_R, n_Z, R, Z, T, V, R_edges, Sigma_g, mu * m_H / k_B, GM,
                                                   rho);
    return cudaGetLastError();
}

} // namespace cdc
