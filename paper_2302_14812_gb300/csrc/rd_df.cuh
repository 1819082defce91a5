// Double-float arithmetic: a value carried as an unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi) / 2), about 48 significant bits, built only from FP32 adds, multiplies and fused
// multiply-adds.  On this GPU FP32 runs 64 times faster than FP64, so a double-float operation
// (6 to 15 FP32 instructions) costs several times less than one FP64 operation.
//
// Building blocks (published error-free transformations):
//   two_sum      Knuth's TwoSum (The Art of Computer Programming, Vol. 2, 4.2.2): s + e = a + b
//                exactly, for any a, b.
//   fast_two_sum Dekker's Fast2Sum (Dekker 1971, "A floating-point technique for extending the
//                available precision"): s + e = a + b exactly when |a| >= |b|.
//   two_prod     the exact product with a fused multiply-add: p = a*b rounded, e = fma(a, b, -p).
// Sums use the "sloppy" double-word addition (TwoSum of the high parts, the low parts added once,
// renormalised by Fast2Sum): its error is bounded by a few units of 2^-48 of |x| + |y|, absolute,
// which is what the differences of neighbouring samples need.  Reciprocal and reciprocal square
// root take the hardware approximation and one Newton-Raphson step evaluated in double-float
// (quadratic convergence: ~2^-22 -> ~2^-44).
//
// Every operation is written with the _rn intrinsics so that the compiler can neither contract a
// product and a sum into one fused multiply-add nor reassociate: the transformations rely on each
// FP32 operation being rounded exactly once, as written.
#pragma once

#include <cuda_runtime.h>

namespace rd {

struct df2 {
    float hi, lo;
};

#ifdef __CUDACC__
__device__ __forceinline__ df2 df_make(float v) { return {v, 0.f}; }

__device__ __forceinline__ float df_round(df2 a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ df2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df2 df_add(df2 a, df2 b)
{
    const df2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df2 df_add_f(df2 a, float b)
{
    const df2 s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df2 df_mul(df2 a, df2 b)
{
    df2 p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df2 df_mul_f(df2 a, float b)
{
    df2 p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// a * 2^k: exact (both parts scaled, no rounding unless they underflow)
__device__ __forceinline__ df2 df_scale2(df2 a, float pow2) { return {__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)}; }

// a * b + c with one renormalisation
__device__ __forceinline__ df2 df_fma(df2 a, df2 b, df2 c)
{
    const df2 p = two_prod(a.hi, b.hi);
    const df2 s = two_sum(p.hi, c.hi);
    float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    t = __fadd_rn(t, __fadd_rn(c.lo, s.lo));
    return fast_two_sum(s.hi, t);
}

// 1 / a: y = rcp.approx(hi), e = 1 - a y (the fused multiply-add makes 1 - hi y exact to its own
// rounding), result y + y e
__device__ __forceinline__ df2 df_rcp(df2 a)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    float e = __fmaf_rn(-a.hi, y, 1.0f);
    e = __fmaf_rn(-a.lo, y, e);
    return fast_two_sum(y, __fmul_rn(y, e));
}

// 1 / sqrt(a), a > 0: y = rsqrt.approx(hi), e = 1 - a y^2 (a y^2 formed in double-float), result
// y + (y/2) e
__device__ __forceinline__ df2 df_rsqrt(df2 a)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    const df2 ayy = df_mul(a, two_prod(y, y));
    const float e = __fsub_rn(__fsub_rn(1.0f, ayy.hi), ayy.lo);
    return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e));
}

// largest integer m with m <= a (|a| < 2^24)
__device__ __forceinline__ int df_floor(df2 a)
{
    const float f = floorf(a.hi);
    int m = (int)f;
    if (f == a.hi && a.lo < 0.f) m -= 1;
    return m;
}

// a >= b for an integer-valued float b
__device__ __forceinline__ bool df_ge(df2 a, float b) { return a.hi > b || (a.hi == b && a.lo >= 0.f); }
#endif

// split of an FP64 value (host or device): hi = nearest float, lo = nearest float to the rest
__host__ __device__ __forceinline__ df2 df_from_double(double v)
{
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

}  // namespace rd
