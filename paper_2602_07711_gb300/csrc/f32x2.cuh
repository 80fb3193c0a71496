// Packed two-lane FP32 arithmetic: add/sub/mul/fma .rn.f32x2 (sm_100 and later) apply one operation to
// both halves of a float2 in a single instruction.  A complex64 value (re, im) and the matching halves
// of two double-float values are float2 pairs, so componentwise complex arithmetic with real
// coefficients takes half the instructions.  Each lane is rounded exactly as the scalar instruction.
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ unsigned long long f2_bits(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 f2_from(unsigned long long u) { return *reinterpret_cast<float2*>(&u); }

__device__ __forceinline__ float2 px_add(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}
__device__ __forceinline__ float2 px_sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}
__device__ __forceinline__ float2 px_mul(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(d);
}
// a * b + c per lane, one rounding
__device__ __forceinline__ float2 px_fma(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from(d);
}
__device__ __forceinline__ float2 px_splat(float s) { return make_float2(s, s); }
