// conv.cuh -- FP64 <-> FP32 conversions on the integer pipe.
#pragma once

#include <cuda_runtime.h>

namespace lg {

// FP64 <-> FP32 conversions on the integer pipe.  GB300 executes the
// conversion instructions on its FP64 pipe (about 1/72 of the FP32 rate), where
// they cost the streaming kernels as much as their arithmetic.  For values in
// the FP32 normal range these take the bit patterns apart with integer
// operations instead, bitwise identical to the conversions (round to nearest,
// ties to even, for FP64 -> FP32: the 29 dropped mantissa bits decide, and a
// carry out of the mantissa raises the exponent, up to infinity); zeros,
// subnormals, overflow, Inf and NaN take the conversion instruction.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    if (e - 897u < 254u) {   // FP32 exponent field e - 896 in 1 .. 254
        const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
        unsigned f = ((e - 896u) << 23) | (unsigned)(m >> 29);
        const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
        f += (rem > 0x10000000u) | ((rem == 0x10000000u) & f);   // the ties to even
        return __uint_as_float(((unsigned)(b >> 32) & 0x80000000u) | f);
    }
    return (float)x;
}

__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned fe = (u >> 23) & 0xffu;
    if (fe - 1u < 254u) {    // FP32 normal
        return __longlong_as_double(
            (long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                        ((unsigned long long)(fe + 896u) << 52) |
                        ((unsigned long long)(u & 0x7fffffu) << 29)));
    }
    return (double)x;
}

}  // namespace lg
