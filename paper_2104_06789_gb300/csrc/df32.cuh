// Float-float ("df32") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, about 44 significant bits, and
// every operation runs on the FP32 pipe. The error-free transformations are
// Knuth's two-sum (TAOCP vol. 2, 4.2.2) and the exact product through a fused
// multiply-add (the rounding error of a * b is fma(a, b, -a*b)); sums and
// products of pairs are renormalised with the fast two-sum that Dekker's
// 1971 paper gives for |a| >= |b|. Each step is written with the _rn
// intrinsics so that the compiler cannot contract or reassociate the
// error terms away.
//
// Used by the per-pixel geometry passes, whose residuals (tenths of a pixel)
// are differences of positions and flows of up to hundreds of pixels: in
// plain FP32 those carry errors of ~1e-5 px, which the likelihood's 1e-5
// relative bound does not allow; in df32 they carry ~1e-11 px.
#pragma once

#include <cuda_runtime.h>

namespace vd {

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_of(float a) { return DF{a, 0.f}; }

// An integer 0 <= i < 2^23 as an exact FP32 value without a conversion
// instruction: 2^23 + i has i in its mantissa bits.
__device__ __forceinline__ float small_int_to_float(int i)
{
    return __fsub_rn(__int_as_float(0x4B000000 | i), 8388608.f);
}

__device__ __forceinline__ float df_to_float(DF a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi);
    const DF t = df_two_sum(a.lo, b.lo);
    const DF u = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ DF df_add(DF a, float b)
{
    const DF s = df_two_sum(a.hi, b);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const DF p = df_two_prod(a.hi, b.hi);
    const float e = fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, p.lo));
    return df_fast_two_sum(p.hi, e);
}

__device__ __forceinline__ DF df_mul(DF a, float b)
{
    const DF p = df_two_prod(a.hi, b);
    return df_fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// a / b: a first quotient in FP32, then two corrections from the df32
// remainder a - q b.
__device__ __forceinline__ DF df_div(DF a, DF b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const DF r1 = df_sub(a, df_mul(b, q1));
    const float q2 = __fdiv_rn(r1.hi, b.hi);
    const DF r2 = df_sub(r1, df_mul(b, q2));
    const float q3 = __fdiv_rn(r2.hi, b.hi);
    return df_add(df_fast_two_sum(q1, q2), q3);
}

// sign of a (hi carries it: lo is zero whenever hi is)
__device__ __forceinline__ bool df_gt0(DF a) { return a.hi > 0.f; }

// a >= c and a <= c for an FP32 c (exact: the difference is formed in df32)
__device__ __forceinline__ bool df_ge(DF a, float c)
{
    const DF d = df_add(a, -c);
    return d.hi >= 0.f;
}

__device__ __forceinline__ bool df_le(DF a, float c)
{
    const DF d = df_add(a, -c);
    return d.hi <= 0.f;
}

// floor(a) for |a| < 2^24
__device__ __forceinline__ int df_floor(DF a)
{
    const float f = floorf(a.hi);
    if (f == a.hi) return (int)f - (a.lo < 0.f ? 1 : 0);
    return (int)f;
}

}  // namespace vd
