// Double-float ("FP32 pair") arithmetic for the few HQL steps whose FP32 rounding would
// be amplified by an ill-conditioned context covariance (the ridge-regularised
// C_YY of Eq. (8) can have a condition number of 1e3..1e4): the covariance
// finalisation and the Cholesky / inverse-factor computation.  A value is hi + lo with
// |lo| <= ulp(hi)/2, about 48 significant bits; every operation runs on the FP32 pipes.
//
// The building blocks are the classic error-free transformations: Knuth's TwoSum,
// Dekker's Fast2Sum (for |a| >= |b|) and the FMA-based TwoProduct; division and square
// root take one Newton correction on top of the FP32 quotient / root, the reciprocal one
// Newton-Raphson step on top of the hardware's approximate reciprocal.
#pragma once

struct df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 df_make(float a) { return {a, 0.0f}; }

// s + e == a + b exactly (Knuth)
__device__ __forceinline__ df32 df_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (Dekker)
__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// p + e == a * b exactly (FMA)
__device__ __forceinline__ df32 df_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ df32 df_add(df32 x, df32 y) {
    df32 s = df_two_sum(x.hi, y.hi);
    df32 t = df_two_sum(x.lo, y.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df32 df_neg(df32 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df32 df_sub(df32 x, df32 y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df32 df_mul(df32 x, df32 y) {
    df32 p = df_two_prod(x.hi, y.hi);
    float c = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    p.lo = __fadd_rn(p.lo, c);
    return df_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df32 df_mul_f(df32 x, float y) {
    df32 p = df_two_prod(x.hi, y);
    p.lo = __fmaf_rn(x.lo, y, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}

// x / y: FP32 quotient, then two correction terms from the exact remainder
__device__ __forceinline__ df32 df_div(df32 x, df32 y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    df32 r = df_sub(x, df_mul_f(y, q1));
    float q2 = __fdiv_rn(r.hi, y.hi);
    r = df_sub(r, df_mul_f(y, q2));
    float q3 = __fdiv_rn(r.hi, y.hi);
    df32 q = df_fast_two_sum(q1, q2);
    return df_add(q, df_make(q3));
}

// 1 / y for y > 0 (normal): Newton-Raphson on the reciprocal, r1 = r0 + r0 (1 - y r0),
// started from the hardware's approximate FP32 reciprocal r0 (about 23 correct bits); one
// step in double-float squares the relative error to about 2^-44.  No division.
__device__ __forceinline__ df32 df_rcp(df32 y) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(y.hi));
    const df32 e = df_sub(df_make(1.0f), df_mul_f(y, r0));
    return df_add(df_make(r0), df_mul_f(e, r0));
}

// sqrt(x) for x > 0: s = sqrtf(hi), then s + (x - s^2) / (2 s)
__device__ __forceinline__ df32 df_sqrt(df32 x) {
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    float s = __fsqrt_rn(x.hi);
    df32 s2 = df_two_prod(s, s);
    df32 r = df_sub(x, s2);
    float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
    return df_fast_two_sum(s, c);
}

// exact conversion of an int (|v| < 2^48) to a pair
__device__ __forceinline__ df32 df_from_int(long long v) {
    float hi = __ll2float_rn(v);
    long long rem = v - (long long)hi;
    return {hi, __ll2float_rn(rem)};
}

__device__ __forceinline__ float df_to_f(df32 x) { return __fadd_rn(x.hi, x.lo); }
