// Conversions between float64 and fp32 by integer operations, with an
// optional power-of-two scale folded into the exponent. On this part the
// float64 pipe runs at 1/64 of the fp32 rate, and a converting instruction
// occupies it like any float64 operation, so kernels that move float64 data
// into a 32- or 16-bit solve convert with these instead.
#pragma once

#include <cuda_runtime.h>

namespace fmp {

// x * 2^k rounded to fp32: to nearest, ties to even (ODD = false), or to odd
// (ODD = true: truncate, then set the last bit when any dropped bit is set; a
// later round-to-nearest-even to a type with at least two fewer fraction
// bits then equals the direct rounding of x * 2^k). Zero and subnormal x, and
// results below 2^-126, give a signed zero; results above the fp32 range give
// infinity; infinities and NaN stay infinities and NaN.
template <bool ODD>
__device__ __forceinline__ float f64_to_f32_scaled(double x, int k) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
    const int ex = static_cast<int>(b >> 52) & 0x7FF;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    int e;
    unsigned f;
    if constexpr (ODD) {
        e = ex - 1023 + 127 + k;
        f = static_cast<unsigned>(m >> 29) | static_cast<unsigned>((m & 0x1FFFFFFFull) != 0);
    } else {
        const unsigned long long r = m + ((1ull << 28) - 1ull) + ((m >> 29) & 1ull);   // 52 -> 23 bits
        e = ex - 1023 + 127 + k + static_cast<int>(r >> 52);   // the carry of a round-up
        f = static_cast<unsigned>(r >> 29) & 0x7FFFFFu;
    }
    unsigned v = (static_cast<unsigned>(e) << 23) | f;
    v = (e <= 0 || ex == 0) ? 0u : v;
    v = e >= 255 ? 0x7F800000u : v;
    v = ex == 0x7FF ? (0x7F800000u | (m != 0 ? 0x400000u : 0u)) : v;
    return __uint_as_float(sign | v);
}

// x * 2^k as float64: exact unless the result leaves the float64 normal range
// (zero below it, infinity above it); fp32 subnormals give zero; infinities
// and NaN stay infinities and NaN.
__device__ __forceinline__ double f32_to_f64_scaled(float x, int k) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFF;
    const unsigned long long sign = static_cast<unsigned long long>(u & 0x80000000u) << 32;
    const unsigned long long mant = static_cast<unsigned long long>(u & 0x7FFFFFu) << 29;
    const int ed = static_cast<int>(e) + 1023 - 127 + k;
    unsigned long long d = sign | (static_cast<unsigned long long>(static_cast<unsigned>(ed) & 0x7FFu) << 52) | mant;
    d = ed <= 0 ? sign : d;
    d = ed >= 0x7FF ? (sign | (0x7FFull << 52)) : d;
    d = e == 0 ? sign : d;
    d = e == 0xFF ? (sign | (0x7FFull << 52) | mant) : d;
    return __longlong_as_double(static_cast<long long>(d));
}

// x rounded to bf16 (to nearest, ties to even) by integer operations, as
// the 16-bit pattern: the same value as rounding to fp32 by odd and then to
// bf16. Results below 2^-126 give a signed zero, above the range infinity;
// NaN stays NaN.
__device__ __forceinline__ unsigned f64_to_bf16_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32);
    const int ex = (int)(hi >> 20) & 0x7FF;
    const int e = ex - 1023 + 127;
    const unsigned m7 = (hi >> 13) & 0x7Fu;
    const unsigned sticky = ((hi & 0xFFFu) | (unsigned)b) != 0u ? 1u : 0u;
    unsigned v = ((unsigned)e << 7) + m7;
    v += ((hi >> 12) & 1u) & (sticky | (m7 & 1u));   // a carry moves into the exponent
    v = (e <= 0 || ex == 0) ? 0u : v;
    v = (e >= 255) ? 0x7F80u : v;
    v = ex == 0x7FF ? (0x7F80u | (((hi & 0xFFFFFu) | (unsigned)b) != 0u ? 0x40u : 0u)) : v;
    return ((hi >> 16) & 0x8000u) | v;
}

// A positive normal s as 2^k * m, m in [1, 2] rounded to fp32 (relative error
// at most 2^-24); anything else gives k = 0, m = 0.
__device__ __forceinline__ void split_pow2(double s, int& k, float& m) {
    const int ex = static_cast<int>(static_cast<unsigned long long>(__double_as_longlong(s)) >> 52);
    const bool ok = ex > 0 && ex < 0x7FF;   // the sign bit makes ex >= 0x800
    k = ok ? ex - 1023 : 0;
    m = ok ? f64_to_f32_scaled<false>(s, -k) : 0.0f;
}

}  // namespace fmp
