// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 44-48 significant bits.  The operations are the error-free transformations of Knuth (two-sum)
// and Dekker (two-product, here via a fused multiply-add), written from their published definitions.
// Used where the solver needs better than FP32 accuracy (true residual, solution accumulator) without
// FP64 arithmetic, whose GB300 throughput is a small fraction of FP32's.
//
// A complex double-float value keeps its two high parts and its two low parts as float2 pairs
// (re.hi, im.hi) and (re.lo, im.lo), so each step of the real algorithms runs on both components in one
// packed two-lane instruction (f32x2.cuh).  Per lane the operation sequence is the scalar one, so the
// results are bit-identical to scalar double-float arithmetic on the real and imaginary parts.
#pragma once
#include <cuda_runtime.h>
#include "f32x2.cuh"

struct df {
    float hi, lo;
};
struct cdf {
    float2 hi, lo;   // (re.hi, im.hi), (re.lo, im.lo)
};

// ---- real double-float ---------------------------------------------------------------------------
__device__ __forceinline__ df df_quick(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return df{s, b - (s - a)};
}
__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return df{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    const df t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_quick(s.hi, s.lo);
    s.lo += t.lo;
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

// ---- packed steps (both lanes at once) -------------------------------------------------------------
// quick two-sum, |a| >= |b| per lane: s + e = a + b exactly
__device__ __forceinline__ void px_quick(float2 a, float2 b, float2& s, float2& e) {
    s = px_add(a, b);
    e = px_sub(b, px_sub(s, a));
}
// two-sum: s + e = a + b exactly
__device__ __forceinline__ void px_two_sum(float2 a, float2 b, float2& s, float2& e) {
    s = px_add(a, b);
    const float2 bb = px_sub(s, a);
    e = px_add(px_sub(a, px_sub(s, bb)), px_sub(b, bb));
}
// two-sum of a and -b: s + e = a - b exactly (negation is exact, so this is two_sum(a, -b) bit for bit)
__device__ __forceinline__ void px_two_diff(float2 a, float2 b, float2& s, float2& e) {
    s = px_sub(a, b);
    const float2 bb = px_sub(s, a);
    e = px_sub(px_sub(a, px_sub(s, bb)), px_add(b, bb));
}
// product of a packed double-float (hi, lo) and a real double-float (sh, sl) broadcast to both lanes
__device__ __forceinline__ cdf px_mul_df(float2 hi, float2 lo, float sh, float sl) {
    const float2 S = px_splat(sh), nS = px_splat(-sh);
    const float2 p = px_mul(hi, S);
    float2 e = px_fma(hi, S, px_mul(hi, nS));   // a.hi b.hi - p, exact
    e = px_fma(hi, px_splat(sl), e);
    e = px_fma(lo, S, e);
    cdf r;
    px_quick(p, e, r.hi, r.lo);
    return r;
}
// product of a packed double-float and a float broadcast to both lanes
__device__ __forceinline__ cdf px_mul_f(float2 hi, float2 lo, float b) {
    const float2 B = px_splat(b);
    const float2 p = px_mul(hi, B);
    float2 e = px_fma(hi, B, px_mul(hi, px_splat(-b)));
    e = px_fma(lo, B, e);
    cdf r;
    px_quick(p, e, r.hi, r.lo);
    return r;
}

// ---- complex double-float --------------------------------------------------------------------------
__device__ __forceinline__ cdf cdf_make(df re, df im) { return cdf{make_float2(re.hi, im.hi), make_float2(re.lo, im.lo)}; }
__device__ __forceinline__ df cdf_re(cdf a) { return df{a.hi.x, a.lo.x}; }
__device__ __forceinline__ df cdf_im(cdf a) { return df{a.hi.y, a.lo.y}; }
__device__ __forceinline__ cdf cdf_zero() { return cdf{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ cdf cdf_from4(float4 v) { return cdf{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 cdf_to4(cdf a) { return make_float4(a.hi.x, a.hi.y, a.lo.x, a.lo.y); }
__device__ __forceinline__ cdf cdf_from_f2(float2 v) { return cdf{v, make_float2(0.f, 0.f)}; }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) {
    cdf s;
    float2 th, tl;
    px_two_sum(a.hi, b.hi, s.hi, s.lo);
    px_two_sum(a.lo, b.lo, th, tl);
    s.lo = px_add(s.lo, th);
    px_quick(s.hi, s.lo, s.hi, s.lo);
    s.lo = px_add(s.lo, tl);
    px_quick(s.hi, s.lo, s.hi, s.lo);
    return s;
}
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) {
    cdf s;
    float2 th, tl;
    px_two_diff(a.hi, b.hi, s.hi, s.lo);
    px_two_diff(a.lo, b.lo, th, tl);
    s.lo = px_add(s.lo, th);
    px_quick(s.hi, s.lo, s.hi, s.lo);
    s.lo = px_add(s.lo, tl);
    px_quick(s.hi, s.lo, s.hi, s.lo);
    return s;
}
// (x, y) -> (-y, x): multiplication by i (exact)
__device__ __forceinline__ cdf cdf_times_i(cdf a) {
    return cdf{make_float2(-a.hi.y, a.hi.x), make_float2(-a.lo.y, a.lo.x)};
}
// a b = a Re(b) + i (a Im(b)); each real product is Dekker's, the sum is one complex double-float add
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    const cdf p = px_mul_df(a.hi, a.lo, b.hi.x, b.lo.x);
    const cdf q = px_mul_df(a.hi, a.lo, b.hi.y, b.lo.y);
    return cdf_add(p, cdf_times_i(q));
}
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) { return px_mul_df(a.hi, a.lo, s.hi, s.lo); }
// a * b with b a plain complex64 value (exact products via FMA)
__device__ __forceinline__ cdf cdf_mul_f2(cdf a, float2 b) {
    const cdf p = px_mul_f(a.hi, a.lo, b.x);
    const cdf q = px_mul_f(a.hi, a.lo, b.y);
    return cdf_add(p, cdf_times_i(q));
}
__device__ __forceinline__ double2 cdf_to_double2(cdf a) { return make_double2(df_to_double(cdf_re(a)), df_to_double(cdf_im(a))); }
__device__ __forceinline__ float2 cdf_round(cdf a) { return px_add(a.hi, a.lo); }
