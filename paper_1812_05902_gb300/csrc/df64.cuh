// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant bits.  GB300 issues
// FP32 at 64 times its FP64 rate, so the 3-20 FP32 instructions of one
// double-float operation are several times cheaper than one FP64 operation.
//
// The primitives are the error-free transformations of Knuth (two-sum),
// Dekker (fast two-sum) and the FMA two-product; add is the "sloppy"
// variant (absolute error ~2^-46 (|a| + |b|)), which is what positions and
// directions need.  Nothing here may be compiled with fast-math.
#pragma once

#include <cuda_runtime.h>

namespace pivbos {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df dfv(float a) { return df{a, 0.0f}; }

__device__ __forceinline__ df df_from_double(double a)
{
    const float hi = __double2float_rn(a);
    const float lo = __double2float_rn(a - (double)hi);
    return df{hi, lo};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (no magnitude condition)
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_add_f(df a, float b)
{
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_sqr(df a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    float e = __fmaf_rn(a.hi, a.hi, -p);
    e = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, e);
    return fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

// 1 / b: FP32 reciprocal refined by one Newton step in double-float
__device__ __forceinline__ df df_rcp(df b)
{
    const float r = __frcp_rn(b.hi);
    // residual 1 - b r, exactly enough in double-float
    const df br = df_mul_f(b, r);
    const df res = df_add_f(df_neg(br), 1.0f);
    return fast_two_sum(r, __fmul_rn(res.hi, r));
}

__device__ __forceinline__ df df_div(df a, df b)
{
    const float r = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const df res = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fmul_rn(res.hi, r);
    return fast_two_sum(q1, q2);
}

// sqrt(a), a >= 0
__device__ __forceinline__ df df_sqrt(df a)
{
    if (a.hi <= 0.0f) return df{0.0f, 0.0f};
    const float x = rsqrtf(a.hi);
    const float y = __fmul_rn(a.hi, x);
    const df y2 = df_sqr(dfv(y));
    const df res = df_sub(a, y2);
    return fast_two_sum(y, __fmul_rn(res.hi, __fmul_rn(0.5f, x)));
}

// 1 / sqrt(a), a > 0: FP32 estimate and one Newton step in double-float
__device__ __forceinline__ df df_rsqrt(df a)
{
    const float x = rsqrtf(a.hi);
    // e = 1 - a x^2 ; result x (1 + e/2)
    const df ax2 = df_mul_f(df_mul_f(a, x), x);
    const df e = df_add_f(df_neg(ax2), 1.0f);
    return fast_two_sum(x, __fmul_rn(__fmul_rn(0.5f, x), e.hi));
}

__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool df_gt(df a, df b) { return df_lt(b, a); }

// floor of a double-float and the (FP32) fraction a - floor(a) in [0, 1)
__device__ __forceinline__ int df_floor(df a, float& frac)
{
    float f = floorf(a.hi);
    float r = __fadd_rn(__fsub_rn(a.hi, f), a.lo);   // exact: a.hi - f is exact for |a.hi| < 2^23
    if (r < 0.0f) {
        f -= 1.0f;
        r += 1.0f;
    } else if (r >= 1.0f) {
        f += 1.0f;
        r -= 1.0f;
    }
    frac = r;
    return (int)f;
}

// compile-time split of a double constant into a double-float
struct df_const {
    float hi, lo;
    constexpr df_const(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
__device__ __forceinline__ df dfc_(const df_const c) { return df{c.hi, c.lo}; }

// sin(pi x), cos(pi x) in double-float for x in half-turns.  Exact reduction
// to a quadrant (q = nearest integer of 2x, r = x - q/2 in [-1/4, 1/4]), the
// Taylor series of sin and cos of theta = pi r (|theta| <= pi/4) in Horner
// form -- double-float for the terms above ~1e-9, FP32 for the tail --
// then an exact quarter-turn rotation.  Absolute error ~1e-14.
__device__ __forceinline__ void df_sincospi(df x, df& s_out, df& c_out)
{
    constexpr df_const kPi(3.14159265358979323846);
    constexpr df_const kS3(-1.0 / 6.0), kS5(1.0 / 120.0), kS7(-1.0 / 5040.0);
    constexpr df_const kC4(1.0 / 24.0), kC6(-1.0 / 720.0), kC8(1.0 / 40320.0);
    const float qf = rintf(2.0f * x.hi);
    const int q = (int)qf;
    const df r = df_add_f(x, -0.5f * qf);
    const df th = df_mul(r, dfc_(kPi));
    const df t2 = df_sqr(th);
    const float f2 = t2.hi;
    // sin(theta)/theta = 1 - t2/3! + t2^2/5! - t2^3/7! + t2^4/9! - t2^5/11! + t2^6/13!
    float ts = 1.0f / 6227020800.0f;                      // 1/13!
    ts = fmaf(ts, -f2, 1.0f / 39916800.0f);               // 1/11! - t2/13!
    ts = fmaf(ts, -f2, 1.0f / 362880.0f);                 // 1/9! - t2/11! + t2^2/13!
    df ps = df_add(df_mul_f(t2, ts), dfc_(kS7));
    ps = df_add(df_mul(t2, ps), dfc_(kS5));
    ps = df_add(df_mul(t2, ps), dfc_(kS3));
    ps = df_add_f(df_mul(t2, ps), 1.0f);
    const df sn = df_mul(th, ps);
    // cos(theta) = 1 - t2/2! + t2^2/4! - t2^3/6! + t2^4/8! - t2^5/10! + t2^6/12! - t2^7/14!
    float tc = 1.0f / 87178291200.0f;                     // 1/14!
    tc = fmaf(tc, -f2, 1.0f / 479001600.0f);              // 1/12! - t2/14!
    tc = fmaf(tc, -f2, 1.0f / 3628800.0f);                // 1/10! - t2/12! + t2^2/14!
    df pc = df_add(df_mul_f(t2, -tc), dfc_(kC8));
    pc = df_add(df_mul(t2, pc), dfc_(kC6));
    pc = df_add(df_mul(t2, pc), dfc_(kC4));
    pc = df_add_f(df_mul(t2, pc), -0.5f);
    const df cn = df_add_f(df_mul(t2, pc), 1.0f);
    switch (q & 3) {
    case 0: s_out = sn; c_out = cn; break;
    case 1: s_out = cn; c_out = df_neg(sn); break;
    case 2: s_out = df_neg(sn); c_out = df_neg(cn); break;
    default: s_out = df_neg(cn); c_out = sn; break;
    }
}

}  // namespace pivbos
