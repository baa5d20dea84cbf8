// Double-float arithmetic: a value carried as an unevaluated sum h + l of two
// FP32 numbers with |l| <= ulp(h) / 2, about 48 significant bits.  The sums
// and products are the classical error-free constructions (Knuth's TwoSum,
// Dekker's FastTwoSum, the fused multiply-add form of the exact product),
// written with explicitly rounded intrinsics so that nothing is fused or
// reassociated.  B300 runs FP32 at many times its FP64 rate, so a kernel
// whose FP64 pipe is its bound can trade each FP64 operation for a handful of
// FP32 ones.  The exponent range is FP32's: values below ~1e-38 flush to
// zero and l loses precision below ~1e-31.
#pragma once
#include <cuda_runtime.h>

namespace cdc {

struct df {
    float h, l;
    df() = default;
    __host__ __device__ constexpr df(float a, float b) : h(a), l(b) {}
    __host__ __device__ constexpr explicit df(int v) : h((float)v), l(0.0f) {}
    __host__ __device__ explicit df(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
    __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// h + l = s + e exactly when |s| >= |e| (FastTwoSum)
__device__ __forceinline__ df df_fast(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return df(h, __fsub_rn(e, __fsub_rn(h, s)));
}
// the sum: TwoSum of the leading parts, the trailing parts added to its
// error, renormalised; error ~2^-47 (|a| + |b|)
__device__ __forceinline__ df operator+(df a, df b)
{
    float s, e;
    df_two_sum(a.h, b.h, s, e);
    return df_fast(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// the product: the exact product of the leading parts (FMA) plus the cross
// terms, renormalised; error ~2^-46 |a b|
__device__ __forceinline__ df operator*(df a, df b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_fast(p, e);
}
__device__ __forceinline__ df &operator+=(df &a, df b) { return a = a + b; }
__device__ __forceinline__ df &operator*=(df &a, df b) { return a = a * b; }

__device__ __forceinline__ df shfl_xor(df v, int o)
{
    return df(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }

// read-only loads of either type through the non-coherent path
__device__ __forceinline__ double ldg(const double *p) { return __ldg(p); }
__device__ __forceinline__ df ldg(const df *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}

} // namespace cdc
