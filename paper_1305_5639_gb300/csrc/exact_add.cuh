// Exact additions into the FP64 long integration without the FP64 pipe's conversions.
// GB300's FP64 pipe is narrow (a few operations per clock per SM), and a plain
// `v + (double)a` spends two FP64 operations per value (the conversion and the add).
// These helpers give bit-identical results with integer instructions doing the
// conversion (FP32 sums) or the whole add (INT32 sums).
#pragma once

#include <cuda_runtime.h>

namespace corr {

// FP32 -> FP64, exact (every float is a double): sign kept, exponent re-biased by
// 1023 - 127 = 896, 23-bit fraction moved to the top of the 52-bit one. Zeros are
// built directly; subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = u & 0x7f800000u;
    if (ex == 0u || ex == 0x7f800000u) {
        if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);  // +-0
        return (double)f;
    }
    const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
}

// v = m 2^(e - 1075) with the hidden bit in m; true (and n set) if v is an integer
// with |v| < 2^52
__device__ __forceinline__ bool dbl_to_i64(unsigned long long b, long long &n) {
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) {  // +-0 (an integer sum has no subnormals)
        n = 0;
        return (b << 1) == 0;
    }
    const int sh = 1075 - e;
    if (sh < 1 || sh > 52) return false;  // |v| >= 2^52 or |v| < 1 (non-zero)
    const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
    if (m & ((1ull << sh) - 1)) return false;  // not an integer
    const long long u = (long long)(m >> sh);
    n = (b >> 63) ? -u : u;
    return true;
}

// exact for |n| < 2^52 (the caller checks)
__device__ __forceinline__ unsigned long long i64_to_dbl(long long n) {
    if (n == 0) return 0ull;
    const unsigned long long s = n < 0 ? (1ull << 63) : 0ull;
    const unsigned long long u = n < 0 ? (unsigned long long)(-n) : (unsigned long long)n;
    const int p = 63 - __clzll((long long)u);  // leading bit, p <= 51
    return s | ((unsigned long long)(p + 1023) << 52) | ((u << (52 - p)) & 0xfffffffffffffull);
}

// v + (a.x, a.y) for an integer-valued long integration (INT8 path): decode each
// double to an int64, add, encode again. Bit-identical to the FP64 add, which is exact
// while |value| < 2^53; an element outside that range, or not an integer, takes the
// FP64 add.
__device__ __forceinline__ double2 add_exact(double2 v, int2 a) {
    long long x, y;
    const unsigned long long bx = (unsigned long long)__double_as_longlong(v.x);
    const unsigned long long by = (unsigned long long)__double_as_longlong(v.y);
    const long long lim = 1ll << 51;
    if (dbl_to_i64(bx, x) && dbl_to_i64(by, y)) {
        x += a.x;
        y += a.y;
        if (x > -lim && x < lim && y > -lim && y < lim)
            return make_double2(__longlong_as_double((long long)i64_to_dbl(x)),
                                __longlong_as_double((long long)i64_to_dbl(y)));
    }
    return make_double2(v.x + (double)a.x, v.y + (double)a.y);
}

// v + (a.x, a.y) for FP32 sums: one FP64 add per value, the conversion in integers
__device__ __forceinline__ double2 add_exact(double2 v, float2 a) {
    return make_double2(v.x + f2d_exact(a.x), v.y + f2d_exact(a.y));
}

}  // namespace corr
