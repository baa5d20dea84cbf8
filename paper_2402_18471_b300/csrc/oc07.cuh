// Ormel & Cuzzi (2007) relative turbulent velocity, shared by the FP64 kernel
// builder and the derivative tables of the adjoint (Sec. 5, Eq. OCVrel).
#pragma once
#include <cuda_runtime.h>

namespace cdc {

// V_rel^2 / V_g^2 from the larger (S1) and smaller (S2) Stokes numbers with
// g1_x = S_x^2 / (1 + S_x), g2_x = S_x^2 / (S_x + d) and d = Re^-1/2: class I
// over slow eddies between t* and t_L and class II over fast eddies between
// t_eta and t*, both particles responding.  St* = clamp(1.6 S1, d, 1).
__device__ __forceinline__ double vrel2_f64(double S1, double S2, double g1_1, double g1_2,
                                            double g2_1, double g2_2, double d)
{
    double Ss = fmin(fmax(1.6 * S1, d), 1.0);
    double dVI = 0.0;
    if (S1 + S2 > 0.0)
        dVI = (S1 - S2) / (S1 + S2) *
              (S1 * S1 / (Ss + S1) - g1_1 - S2 * S2 / (Ss + S2) + g1_2);
    double dVII = 2.0 * (Ss - d) + S1 * S1 / (S1 + Ss) - g2_1 + S2 * S2 / (S2 + Ss) - g2_2;
    return fmax(dVI + dVII, 0.0);
}

// d(V_rel^2 / V_g^2) / d(d) at fixed Stokes numbers: the explicit d of class
// II (its lower limit and the g2 terms) plus, where St* is clamped to d, the
// dependence through St*.  Zero where the sum is clamped at 0.
__device__ __forceinline__ double dvrel2_dd_f64(double S1, double S2, double d)
{
    const double a16 = 1.6 * S1;
    double Ss = fmin(fmax(a16, d), 1.0);
    double dVI = 0.0;
    if (S1 + S2 > 0.0)
        dVI = (S1 - S2) / (S1 + S2) *
              (S1 * S1 / (Ss + S1) - S1 * S1 / (1.0 + S1) - S2 * S2 / (Ss + S2) + S2 * S2 / (1.0 + S2));
    const double dVII = 2.0 * (Ss - d) + S1 * S1 / (S1 + Ss) - S1 * S1 / (S1 + d) +
                        S2 * S2 / (S2 + Ss) - S2 * S2 / (S2 + d);
    if (!(dVI + dVII > 0.0)) return 0.0;
    const double q1 = S1 / (S1 + d), q2 = S2 / (S2 + d);
    double r = -2.0 + q1 * q1 + q2 * q2;
    if (a16 < d && d < 1.0) {
        const double p1 = S1 / (Ss + S1), p2 = S2 / (Ss + S2);
        if (S1 + S2 > 0.0) r += (S1 - S2) / (S1 + S2) * (p2 * p2 - p1 * p1);
        r += 2.0 - p1 * p1 - p2 * p2;
    }
    return r;
}

} // namespace cdc
