// df.cuh -- double-float arithmetic: a value carried as the unevaluated sum
// hi + lo of two FP32 numbers (about 48 significant bits), on the FP32 pipe.
#pragma once

#include <cuda_runtime.h>

namespace lg {

// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, FMA-based
// TwoProd).  The explicit _rn intrinsics keep the compiler from contracting
// or re-associating them.
struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// x + y; absolute error about 2^-47 (|x| + |y|).
__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    const dfl s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// x * y; relative error about 2^-46.
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_split(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// x * c for an FP32 constant c.
__device__ __forceinline__ dfl df_mul_f(dfl x, float c)
{
    const float p = __fmul_rn(x.hi, c);
    return df_fast_two_sum(p, __fmaf_rn(x.lo, c, __fmaf_rn(x.hi, c, -p)));
}

__device__ __forceinline__ dfl df_neg(dfl x) { return dfl{-x.hi, -x.lo}; }

}  // namespace lg
