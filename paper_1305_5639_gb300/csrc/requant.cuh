// 8-bit re-packing of channelised samples (shared by the F-engine kernels):
// q = clamp(rint(S * scale), -127, 127), ties to even, and the exact expansion of
// offset-binary code pairs into the planar FP16 layout.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_common.cuh"

namespace corr {

// 1.5 * 2^23: adding it to |v| <= 2^22 rounds v to the nearest integer (ties to
// even, the FP32 adder's rounding) and leaves that integer in the low mantissa bits.
constexpr float kMagic = 12582912.0f;

// Re-pack to int8: q = clamp(rint(S * scale), -127, 127), round half to even.
// One FMA adds the magic constant M to the product, which rounds it to an integer
// kept in the low mantissa bits (rint of the exact product); the clamp is then taken
// on M + q, which is monotonic in the product for every input, so clamping after
// rounding equals rounding after clamping. The low byte of each result is the code:
// two's complement (M = 1.5 * 2^23) or offset binary q + 128 (M + 128, OB).
template <bool OB>
__device__ __forceinline__ uint32_t pack_q(float2 v, float sc) {
    constexpr float M = OB ? kMagic + 128.0f : kMagic;
    float2 t = f2_fma(v, make_float2(sc, sc), make_float2(M, M));
    t = make_float2(fminf(fmaxf(t.x, M - 127.0f), M + 127.0f), fminf(fmaxf(t.y, M - 127.0f), M + 127.0f));
    return __byte_perm(__float_as_uint(t.x), __float_as_uint(t.y), 0x0040);
}

// Two complex offset-binary codes [re0 im0 re1 im1] (code = q + 128) -> FP16 pairs
// (q_re0, q_re1) and (q_im0, q_im1), exactly: the half with bits 0x64uu is 1024 + u.
__device__ __forceinline__ void ob_codes_to_f16_planes(uint32_t u, uint32_t &re, uint32_t &im) {
    uint32_t hr = __byte_perm(u, 0x64646464u, 0x4240), hi = __byte_perm(u, 0x64646464u, 0x4341);
    const __half2 k1152 = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));
    __half2 r = __hsub2(*reinterpret_cast<__half2 *>(&hr), k1152);
    __half2 m = __hsub2(*reinterpret_cast<__half2 *>(&hi), k1152);
    re = *reinterpret_cast<uint32_t *>(&r);
    im = *reinterpret_cast<uint32_t *>(&m);
}

}  // namespace corr
