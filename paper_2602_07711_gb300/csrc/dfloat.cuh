// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 44-48 significant bits.  The operations are the error-free transformations of Knuth (two-sum)
// and Dekker (two-product, here via a fused multiply-add), written from their published definitions.
// Used where the solver needs better than FP32 accuracy (true residual, solution accumulator) without
// FP64 arithmetic, whose GB300 throughput is a small fraction of FP32's.
#pragma once
#include <cuda_runtime.h>

struct df {
    float hi, lo;
};
struct cdf {
    df re, im;
};

__device__ __forceinline__ df df_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return df{s, b - (s - a)};
}
__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return df{s, (a - (s - bb)) + (b - bb)};
}
// Sum of two double-float values with one two-sum (of the high parts); the low parts are added in FP32.
// The absolute error stays below about 2^-44 (|a| + |b|), which is what the residual and the right-hand
// side need: their cancellations leave results no smaller than ~1e-11 of the operands.
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_quick(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_quick(p, e);
}
__device__ __forceinline__ df df_from_double(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ cdf cdf_zero() { return cdf{df{0.f, 0.f}, df{0.f, 0.f}}; }
__device__ __forceinline__ cdf cdf_from4(float4 v) { return cdf{df{v.x, v.z}, df{v.y, v.w}}; }
__device__ __forceinline__ float4 cdf_to4(cdf a) { return make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo); }
__device__ __forceinline__ cdf cdf_from_f2(float2 v) { return cdf{df{v.x, 0.f}, df{v.y, 0.f}}; }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    return cdf{df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return cdf{df_mul(a.re, s), df_mul(a.im, s)}; }
// a * b with b a plain complex64 value (exact products via FMA)
__device__ __forceinline__ cdf cdf_mul_f2(cdf a, float2 b) {
    return cdf{df_sub(df_mulf(a.re, b.x), df_mulf(a.im, b.y)), df_add(df_mulf(a.re, b.y), df_mulf(a.im, b.x))};
}
__device__ __forceinline__ double2 cdf_to_double2(cdf a) { return make_double2(df_to_double(a.re), df_to_double(a.im)); }
__device__ __forceinline__ float2 cdf_round(cdf a) { return make_float2(a.re.hi + a.re.lo, a.im.hi + a.im.lo); }
