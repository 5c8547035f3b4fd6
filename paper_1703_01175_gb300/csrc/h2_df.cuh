// Double-float arithmetic on the FP32 pipes: a value is the unevaluated sum
// hi + lo of two floats (48-bit significand). Products are split exactly with
// an FMA (TwoProd) and running sums carry their rounding error in a second
// float (TwoSum, Knuth), as in the compensated dot product of Ogita, Rump &
// Oishi (2005). Every operation uses the _rn intrinsics, which the compiler
// never contracts into other FMAs, so the error-free steps stay exact.
#pragma once

#include <cuda_runtime.h>

namespace h2 {

static __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, c) += (ah + al) (bh + bl), product split exactly, sum compensated
static __device__ __forceinline__ void df_mac(float &s, float &c, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float t, q;
    two_sum(s, p, t, q);
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

static __device__ __forceinline__ double df_to_d(float s, float c) { return (double)s + (double)c; }

static __device__ __forceinline__ float2 d_to_df(double d)
{
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

// renormalise (s, c) so that |lo| <= ulp(hi) / 2
static __device__ __forceinline__ float2 df_norm(float s, float c)
{
    float h, l;
    two_sum(s, c, h, l);
    return make_float2(h, l);
}

// (s, c) += a (bh + bl) for a plain float a
static __device__ __forceinline__ void df_macf(float &s, float &c, float a, float bh, float bl)
{
    const float p = __fmul_rn(a, bh);
    float e = __fmaf_rn(a, bh, -p);
    e = __fmaf_rn(a, bl, e);
    float t, q;
    two_sum(s, p, t, q);
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

}  // namespace h2
