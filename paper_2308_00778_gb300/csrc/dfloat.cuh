// dfloat.cuh -- double-float helpers: sums and products carried as pairs of binary32.
#pragma once

namespace gsr {

// s + e = a + b exactly (Knuth's two-sum); explicit roundings, no contraction
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// (s, c) += a * (x.x + x.y): the leading product split exactly with an FMA
// (p + pe = a * x.x), the small product a * x.y and all error terms go to c.
__device__ __forceinline__ void acc_term(float a, float2 x, float &s, float &c)
{
    const float p = __fmul_rn(a, x.x);
    const float pe = __fmaf_rn(a, x.x, -p);
    const float q = __fmul_rn(a, x.y);
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, __fadd_rn(pe, q)));
}

// a binary64 value as the pair (hi, lo) of binary32 with hi + lo ~ v to about 2^-48
__device__ __forceinline__ float2 split_double(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

}  // namespace gsr
