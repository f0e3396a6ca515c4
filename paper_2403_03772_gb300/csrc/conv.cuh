// conv.cuh -- FP64 <-> FP32 conversions on the integer pipe.
#pragma once

#include <cuda_runtime.h>

namespace lg {

// FP64 <-> FP32 conversions on the integer pipe.  GB300 executes the
// conversion instructions on its FP64 pipe (about 1/72 of the FP32 rate), where
// they cost the streaming kernels as much as their arithmetic.  These take the
// bit patterns apart with integer operations only, for every input, and give
// the instructions' results bit for bit (a NaN gives a quiet NaN of the same
// sign).  FP64 -> FP32 rounds to nearest, ties to even: in the FP32 normal
// range the 29 dropped mantissa bits decide, and a carry out of the mantissa
// raises the exponent, up to infinity; below that range the significand is
// shifted onto units of 2^-149 (an FP32 subnormal) with the same rounding;
// |x| >= 2^128 gives infinity.  FP32 -> FP64 is exact (FP32 subnormals are
// normalised).
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    unsigned f;
    if (e - 897u < 254u) {            // FP32 exponent field e - 896 in 1 .. 254
        f = ((e - 896u) << 23) | (unsigned)(m >> 29);
        const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);
        f += (rem > 0x10000000u) | ((rem == 0x10000000u) & f);   // the ties to even
    } else if (e >= 1151u) {          // beyond the FP32 range, or Inf / NaN
        f = (e == 2047u && m != 0ull) ? 0x7fc00000u : 0x7f800000u;
    } else {                          // an FP32 subnormal or zero (e <= 896)
        const unsigned sh = 926u - e; // the significand's shift onto 2^-149 units, >= 30
        if (sh > 54u) {
            f = 0u;                   // below half of 2^-149 (and FP64 subnormals)
        } else {
            const unsigned long long M = m | (1ull << 52);
            f = (unsigned)(M >> sh);
            const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
            f += (rem > half) | ((rem == half) & (f & 1u));
        }
    }
    return __uint_as_float(sign | f);
}

__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned fe = (u >> 23) & 0xffu, fm = u & 0x7fffffu;
    unsigned long long d;
    if (fe - 1u < 254u) {             // FP32 normal
        d = ((unsigned long long)(fe + 896u) << 52) | ((unsigned long long)fm << 29);
    } else if (fe == 255u) {          // Inf / NaN
        d = (0x7ffull << 52) | ((unsigned long long)fm << 29);
    } else if (fm == 0u) {            // zero
        d = 0ull;
    } else {                          // FP32 subnormal fm 2^-149, normalised
        const int c = __clz(fm);      // 9 .. 31
        d = ((unsigned long long)(905 - c) << 52) |
            (((unsigned long long)fm << (21 + c)) & 0xFFFFFFFFFFFFFull);
    }
    return __longlong_as_double((long long)(sign | d));
}

}  // namespace lg
