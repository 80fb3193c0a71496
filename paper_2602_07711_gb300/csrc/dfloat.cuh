// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 44-48 significant bits.  The operations are the error-free transformations of Knuth (two-sum)
// and Dekker (two-product, here via a fused multiply-add), written from their published definitions.
// Used where the solver needs better than FP32 accuracy (true residual, solution accumulator) without
// FP64 arithmetic, whose GB300 throughput is a small fraction of FP32's.
//
// A complex double-float value keeps its two high parts and its two low parts as pairs, hi = (re.hi,
// im.hi) and lo = (re.lo, im.lo) (the float4 layout it is stored in), so that every step of an operation
// on the real and the imaginary part is one packed f32x2 instruction.  The results equal those of the
// same steps done part by part in scalar FP32.
#pragma once
#include <cuda_runtime.h>
#include "packed.cuh"

struct df {
    float hi, lo;
};
struct cdf {
    float2 hi, lo;
};

// scalar forms (host-side constants and the few scalar uses)
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
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_quick(p, e);
}
__device__ __forceinline__ df df_from_double(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// ---- complex, packed --------------------------------------------------------------------------
__device__ __forceinline__ cdf cdf_zero() { return cdf{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ cdf cdf_from4(float4 v) { return cdf{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 cdf_to4(cdf a) { return make_float4(a.hi.x, a.hi.y, a.lo.x, a.lo.y); }
__device__ __forceinline__ cdf cdf_from_f2(float2 v) { return cdf{v, make_float2(0.f, 0.f)}; }
__device__ __forceinline__ cdf cdf_neg(cdf a) { return cdf{make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)}; }

// quick two-sum of pairs, |s| >= |e| per half: (s + e, e - ((s + e) - s))
__device__ __forceinline__ cdf cdf_quick(float2 s, float2 e) {
    const float2 h = add2(s, e);
    return cdf{h, sub2(e, sub2(h, s))};
}
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) {
    const float2 s = add2(a.hi, b.hi);
    const float2 bb = sub2(s, a.hi);
    float2 e = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));   // two-sum error of the high parts
    e = add2(e, add2(a.lo, b.lo));
    return cdf_quick(s, e);
}
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) {
    // a + (-b), negation exact: the same steps as cdf_add with the signs folded into subtractions
    const float2 s = sub2(a.hi, b.hi);
    const float2 bb = sub2(s, a.hi);
    float2 e = sub2(sub2(a.hi, sub2(s, bb)), add2(b.hi, bb));      // (a - (s - bb)) + (-b - bb)
    e = add2(e, sub2(a.lo, b.lo));
    return cdf_quick(s, e);
}
// Dekker product of the pairs x (double-float) by the broadcast double-float scalar s, carried with
// pn = -p = -(x.hi s.hi) so that no separate negation is needed: e = x.hi s.hi - p (exact), then the
// cross terms, then the quick two-sum of p and e.
__device__ __forceinline__ cdf cdf_scale(cdf a, df s) {
    const float2 pn = mul2(a.hi, bc2(-s.hi));
    float2 e = fma2(a.hi, bc2(s.hi), pn);
    e = fma2(a.hi, bc2(s.lo), e);
    e = fma2(a.lo, bc2(s.hi), e);
    const float2 h = sub2(e, pn);                  // p + e
    return cdf{h, sub2(e, add2(h, pn))};           // e - ((p + e) - p)
}
// the pair (x0 y, x1 y) of a double-float scalar y = (yh, yl) times the pairs xh, xl of two double-floats
__device__ __forceinline__ cdf cdf_pair_mul(float2 xh, float2 xl, float yh, float yl) {
    const float2 pn = mul2(xh, bc2(-yh));
    float2 e = fma2(xh, bc2(yh), pn);
    e = fma2(bc2(yh), xl, e);
    e = fma2(bc2(yl), xh, e);
    const float2 h = sub2(e, pn);
    return cdf{h, sub2(e, add2(h, pn))};
}
// complex product: (a.re b.re - a.im b.im, a.re b.im + a.im b.re) as X + (-1, 1) Y with
// X = a.re (b.re, b.im) and Y = a.im (b.im, b.re), each a pair of Dekker products
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
    const cdf X = cdf_pair_mul(b.hi, b.lo, a.hi.x, a.lo.x);
    cdf Y = cdf_pair_mul(swap2(b.hi), swap2(b.lo), a.hi.y, a.lo.y);
    Y.hi.x = -Y.hi.x;
    Y.lo.x = -Y.lo.x;
    return cdf_add(X, Y);
}
// a * b with b a plain complex64 value (exact products via FMA)
__device__ __forceinline__ cdf cdf_mul_f2(cdf a, float2 b) {
    const cdf X = cdf_pair_mul(b, make_float2(0.f, 0.f), a.hi.x, a.lo.x);
    cdf Y = cdf_pair_mul(swap2(b), make_float2(0.f, 0.f), a.hi.y, a.lo.y);
    Y.hi.x = -Y.hi.x;
    Y.lo.x = -Y.lo.x;
    return cdf_add(X, Y);
}
// ---- unnormalised pairs: compensated sums of many double-float terms --------------------------
// Within one long sum the renormalisation after every step can be left out: the high parts are summed in
// FP32 with the exact two-sum error of every addition (and the exact FMA error of every product), and those
// errors, together with the terms' low parts, are summed in a second FP32 accumulator.  hi + lo is the
// value (lo is not bounded by ulp(hi)); the absolute error stays near (number of terms) x 2^-48 x the sum
// of the terms' magnitudes, the behaviour of the compensated summation and dot product of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005).  Used by the sixth-order residual,
// whose ~40 additions per point would otherwise each end in a quick two-sum.
__device__ __forceinline__ cdf cp_add(cdf a, cdf b) {
    const float2 s = add2(a.hi, b.hi);
    const float2 bb = sub2(s, a.hi);
    const float2 t = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
    return cdf{s, add2(add2(a.lo, b.lo), t)};
}
__device__ __forceinline__ cdf cp_sub(cdf a, cdf b) {
    const float2 s = sub2(a.hi, b.hi);
    const float2 bb = sub2(s, a.hi);
    const float2 t = sub2(sub2(a.hi, sub2(s, bb)), add2(b.hi, bb));   // (a - (s - bb)) + (-b - bb)
    return cdf{s, add2(sub2(a.lo, b.lo), t)};
}
// a + b with b a plain complex64 value
__device__ __forceinline__ cdf cp_add_f2(cdf a, float2 b) {
    const float2 s = add2(a.hi, b);
    const float2 bb = sub2(s, a.hi);
    const float2 t = add2(sub2(a.hi, sub2(s, bb)), sub2(b, bb));
    return cdf{s, add2(a.lo, t)};
}
// a times the float k: the high parts' product with its exact FMA error, the low parts times k
__device__ __forceinline__ cdf cp_mulk(cdf a, float k) {
    const float2 p = mul2(a.hi, bc2(k));
    const float2 t = make_float2(fmaf(a.hi.x, k, -p.x), fmaf(a.hi.y, k, -p.y));
    return cdf{p, fma2(a.lo, bc2(k), t)};
}
// a times the double-float scalar s
__device__ __forceinline__ cdf cp_mul(cdf a, df s) {
    const float2 p = mul2(a.hi, bc2(s.hi));
    float2 t = make_float2(fmaf(a.hi.x, s.hi, -p.x), fmaf(a.hi.y, s.hi, -p.y));
    t = fma2(a.hi, bc2(s.lo), t);
    return cdf{p, fma2(a.lo, bc2(s.hi), t)};
}
// ---- FP64 <-> double-float on the bit patterns --------------------------------------------------
// GB300's FP64 and FP64-conversion pipes run at a small fraction of its FP32 and integer rate (a stream of
// double -> double-float conversions ran at a third of HBM bandwidth on them), so the conversions of the
// solver's vectors are formed on the IEEE bit patterns with integer and FP32 instructions.  Both give the
// same bits as the FP64 forms (float)v, (float)(v - (double)(float)v) and (double)hi + (double)lo; values
// outside the ranges stated below, rare in a solve, take those FP64 forms.
//
// split: hi = v rounded to nearest even on the 52-bit mantissa; v - hi = d 2^(e-52) exactly with d an
// integer of at most 29 bits, and lo = d rounded once to a float (two exact pieces of d joined by one fma)
// times 2^(e-52).  Fast path for 2^-74 <= |v| < 2^127 (so that 2^(e-52) is a normal float).
// The FP64 forms for the rare values outside the fast paths live in functions of their own (not inlined),
// so that the compiler cannot predicate their FP64 instructions into the common path.
static __device__ __noinline__ float2 df_split_fp64(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
static __device__ __noinline__ double df_widen_fp64(float f) { return (double)f; }
static __device__ __noinline__ double df_join_fp64(float hi, float lo) { return (double)hi + (double)lo; }

__device__ __forceinline__ float2 df_split(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(b >> 32);
    if ((b << 1) == 0ull) return make_float2(__uint_as_float(hw & 0x80000000u), 0.f);   // +-0
    const int e = (int)((hw >> 20) & 0x7FFu) - 1023;
    if (e < -74 || e > 126) return df_split_fp64(v);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    const unsigned mh = (unsigned)(m >> 29);                    // the top 23 mantissa bits
    const unsigned r = (unsigned)(m & 0x1FFFFFFFull);           // the 29 bits below them
    const unsigned up = (r > 0x10000000u || (r == 0x10000000u && (mh & 1u))) ? 1u : 0u;
    const unsigned sign = hw & 0x80000000u;
    const float hi = __uint_as_float(sign | ((((unsigned)(e + 127)) << 23) + mh + up));   // a carry bumps e
    const int d = (int)r - (int)(up << 29);                     // v - hi in units of 2^(e-52), |d| <= 2^28
    const int d1 = d >> 16, d0 = d & 0xFFFF;                     // d = 65536 d1 + d0, |d1| <= 2^12
    const float f1 = __int_as_float(0x4B400000 + d1) - 12582912.f;   // exact: 1.5 2^23 + d1
    const float f0 = __int_as_float(0x4B000000 + d0) - 8388608.f;    // exact: 2^23 + d0
    const float l = fmaf(f1, 65536.f, f0);                       // d, rounded once
    const float sc = __uint_as_float(((unsigned)(e - 52 + 127)) << 23);   // 2^(e-52), normal for e >= -74
    return make_float2(hi, (sign ? -l : l) * sc);
}
// exact float -> double on the bit pattern (normal floats and zero; subnormal, infinite and NaN floats
// take the conversion)
__device__ __forceinline__ double df_widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xFFu;
    if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));   // +-0
    if (ef == 0u || ef == 255u) return df_widen_fp64(f);
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(ef - 127u + 1023u) << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}
// hi + lo rounded to nearest even, on the bit patterns: with hi normal and lo normal, G = e(hi) - e(lo) >= 1,
// the sum is hi's double pattern plus or minus k, k = |lo| in units of hi's double ulp 2^(e(hi)-52): exact
// when G <= 29, else rounded to nearest even (hi's double mantissa ends in 29 zero bits, so the parity of
// the result is that of k).  While the result stays in hi's binade the patterns are linear in the value;
// a carry or borrow across it, a zero or subnormal part, and G < 1 take the FP64 addition.
__device__ __forceinline__ double df_join(float hi, float lo) {
    const unsigned uh = __float_as_uint(hi), ul = __float_as_uint(lo);
    const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
    if ((ul << 1) == 0u) return df_widen(hi);                           // lo = +-0
    const int G = eh - el;
    // (a power-of-two hi with lo of the other sign rounds on the finer grid below it: FP64 as well)
    if (eh == 0 || eh == 255 || el == 0 || el == 255 || G < 1 ||
        (((uh ^ ul) & 0x80000000u) && (uh & 0x7FFFFFu) == 0u))
        return df_join_fp64(hi, lo);
    const unsigned long long bh = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                  ((unsigned long long)(eh - 127 + 1023) << 52) |
                                  ((unsigned long long)(uh & 0x7FFFFFu) << 29);
    const unsigned ml = (ul & 0x7FFFFFu) | 0x800000u;                   // lo's 24-bit significand
    unsigned long long k;
    if (G <= 29) {
        k = (unsigned long long)ml << (29 - G);
    } else {
        const int sh = G - 29;
        if (sh >= 25) {
            k = 0ull;                                                   // |lo| below half an ulp
        } else {
            const unsigned q = ml >> sh, rem = ml & ((1u << sh) - 1u), half = 1u << (sh - 1);
            k = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
        }
    }
    const unsigned long long r = ((uh ^ ul) & 0x80000000u) ? bh - k : bh + k;
    if ((r ^ bh) >> 52) return df_join_fp64(hi, lo);                   // left hi's binade
    return __longlong_as_double((long long)r);
}
__device__ __forceinline__ float4 split4_bits(double2 v) {
    const float2 re = df_split(v.x), im = df_split(v.y);
    return make_float4(re.x, im.x, re.y, im.y);
}
__device__ __forceinline__ double2 cdf_to_double2(cdf a) {
    return make_double2(df_join(a.hi.x, a.lo.x), df_join(a.hi.y, a.lo.y));
}
// the same value by two FP64 additions: cheaper in kernels whose FP64 pipe is otherwise idle and whose
// integer issue is the limit (the sixth-order right-hand side)
__device__ __forceinline__ double2 cdf_to_double2_fp64(cdf a) {
    return make_double2(df_widen(a.hi.x) + df_widen(a.lo.x), df_widen(a.hi.y) + df_widen(a.lo.y));
}
__device__ __forceinline__ double2 df4_to_double2(float4 v) {
    return make_double2(df_join(v.x, v.z), df_join(v.y, v.w));
}
// |v|^2 of a complex64 value accumulated into a per-thread compensated FP32 sum (Kahan)
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c, t = s + y;
    c = (t - s) - y;
    s = t;
}
__device__ __forceinline__ float2 cdf_round(cdf a) { return add2(a.hi, a.lo); }
