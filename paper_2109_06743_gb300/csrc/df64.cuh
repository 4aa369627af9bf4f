// Double-float ("df64") arithmetic on the FP32 pipe: a value is hi + lo with
// two floats. On GB300 the FP64 pipe runs at ~1/58 of the FP32 pipe, so the
// per-cell arithmetic of the moment fit that needs more than FP32 precision
// uses these error-free transformations instead (about 44 significant bits):
//   TwoSum (Knuth): s = a + b exactly as s + e,
//   TwoProduct with FMA: p = a * b exactly as p + e.
// exp is evaluated as 2^k exp(r), |r| <= ln2/2, with the Taylor series of
// exp(r) to degree 13 in double-float arithmetic (truncation < 1e-17).
// The transformations use the _rn intrinsics, which the compiler never
// contracts into fused multiply-adds (contraction would break them).
#pragma once

#include <cuda_runtime.h>

namespace vl {

struct df2 {
    float hi, lo;
};

__device__ __forceinline__ df2 df2_make(float h, float l) { return {h, l}; }
__device__ __forceinline__ df2 df2_f(float x) { return {x, 0.f}; }
// FP64 -> df (FP64 pipe: use outside inner loops only)
__device__ __forceinline__ df2 df2_d(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df2_to_d(df2 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df2 df2_qtwo_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df2 df2_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df2 df2_add(df2 a, df2 b) {
    df2 s = df2_two_sum(a.hi, b.hi);
    df2 t = df2_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df2_qtwo_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df2_qtwo_sum(s.hi, s.lo);
}
__device__ __forceinline__ df2 df2_neg(df2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df2 df2_sub(df2 a, df2 b) { return df2_add(a, df2_neg(b)); }
__device__ __forceinline__ df2 df2_mul(df2 a, df2 b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df2_qtwo_sum(p, e);
}
__device__ __forceinline__ df2 df2_mulf(df2 a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df2_qtwo_sum(p, e);
}
// a / b: FP32 quotient, then one correction from the double-float remainder
__device__ __forceinline__ df2 df2_div(df2 a, df2 b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df2 r = df2_sub(a, df2_mulf(b, q1));
    return df2_qtwo_sum(q1, __fdiv_rn(r.hi, b.hi));
}
// a * b + c
__device__ __forceinline__ df2 df2_fma(df2 a, df2 b, df2 c) { return df2_add(df2_mul(a, b), c); }

// 1 / n! for n = 0..13 as double-float pairs (nearest float, then the
// nearest float of the remainder, from the exact rational value)
static __constant__ float kInvFact[14][2] = {
    {1.000000000e+00f, 0.000000000e+00f},
    {1.000000000e+00f, 0.000000000e+00f},
    {5.000000000e-01f, 0.000000000e+00f},
    {1.666666716e-01f, -4.967053879e-09f},
    {4.166666791e-02f, -1.241763470e-09f},
    {8.333333768e-03f, -4.346172033e-10f},
    {1.388888923e-03f, -3.363109444e-11f},
    {1.984127011e-04f, -2.725596875e-12f},
    {2.480158764e-05f, -3.406996094e-13f},
    {2.755731884e-06f, 3.793571224e-14f},
    {2.755731998e-07f, -7.575112209e-15f},
    {2.505210794e-08f, 4.417623045e-16f},
    {2.087675588e-09f, 1.108283915e-16f},
    {1.605904437e-10f, -5.352526512e-18f}};

static __device__ __noinline__ df2 df2_exp(df2 x) {
    const float kInvLn2 = 1.4426950408889634f;
    const df2 ln2 = {6.931471825e-01f, -1.904654210e-09f};
    if (!(x.hi > -87.0f)) return {0.f, 0.f};
    if (!(x.hi < 88.0f)) return {__int_as_float(0x7f800000), 0.f};
    const float k = rintf(x.hi * kInvLn2);
    // r = x - k ln2, k ln2 formed exactly (TwoProduct) before subtracting
    float p = __fmul_rn(k, ln2.hi);
    float e = fmaf(k, ln2.hi, -p);
    df2 kl = df2_qtwo_sum(p, fmaf(k, ln2.lo, e));
    df2 r = df2_sub(x, kl);
    df2 s = {kInvFact[13][0], kInvFact[13][1]};
#pragma unroll
    for (int n = 12; n >= 0; --n) s = df2_fma(s, r, df2{kInvFact[n][0], kInvFact[n][1]});
    const int ki = (int)k;
    return {ldexpf(s.hi, ki), ldexpf(s.lo, ki)};
}

}  // namespace vl
