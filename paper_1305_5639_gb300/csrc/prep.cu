// Complex float channelised data -> planar FP16 operands for the TMA X-engine.
//   plain (2 planes):  h = fp16(x 2^e) for Re and Im
//   hi/lo (4 planes):  h = fp16(x 2^e), l = fp16(x 2^e - h) for Re and Im, so that
//                      x 2^e = h + l to about 2^-22 relative and
//                      x_i conj(x_j) ~ (h_i conj(h_j) + h_i conj(l_j) + l_i conj(h_j)) 2^-(e_i + e_j)
// (the l l term, ~2^-22 relative, is dropped). x 2^e - h is exact in FP32.
//
// Range: one power of two 2^e per (channel, input) row, chosen from the row's
// largest component so that it lands in [2^14, 2^15): FP16 then neither
// overflows (above 65504) nor loses the low part l to its subnormal range,
// whatever the data's magnitude. The scale is exact; the X-engine epilogue undoes
// it (V_ij times 2^-e_i 2^-e_j), and the reciprocals 2^-e are written to
// row_scale [chan][input].
//
// Layout [chan][plane][input][Kp] (planes Re_h, Im_h (, Re_l, Im_l)), Kp = the
// spectra rounded up to a multiple of 8 so that every row starts on a 16-byte
// boundary (a TMA requirement); the tail is written as zeros. Rows of up to 4096
// spectra are held in the registers of one CTA (k_to_planar_row); longer rows take
// one warp per row, a pass for the maximum and then the conversion (the row re-read
// from L1/L2). HBM sees 8 B read and 4 B (plain) or 8 B (hi/lo) written per complex
// sample.
#include <cuda_fp16.h>

#include "internal.h"

namespace corr {
namespace {

constexpr int kWarps = 8;

// 4 consecutive spectra [s, s + 4) of one row as (re0 im0 re1 im1), (re2 im2 re3 im3),
// zero outside [0, K); VEC: the row start is 16-byte aligned (K even).
template <bool VEC>
__device__ __forceinline__ void load_quad(const float2 *row, int s, int K, float4 &a, float4 &b) {
    if (VEC && s + 4 <= K) {
        a = __ldg(reinterpret_cast<const float4 *>(row + s));
        b = __ldg(reinterpret_cast<const float4 *>(row + s + 2));
        return;
    }
    float2 v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = s + e < K ? __ldg(row + s + e) : make_float2(0.f, 0.f);
    a = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    b = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}

__device__ __forceinline__ float amax4(const float4 &a) {
    return fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }

template <int NPL, bool VEC>
__global__ void __launch_bounds__(32 * kWarps) k_to_planar(const float2 *__restrict__ X, uint2 *__restrict__ out,
                                                           float *__restrict__ row_scale, long long n_rows, int n_in,
                                                           int K, int Kp) {
    const int lane = threadIdx.x & 31;
    const int nq = Kp / 4;  // quads of spectra per padded row
    for (long long row = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); row < n_rows;
         row += (long long)gridDim.x * kWarps) {
        const float2 *x = X + row * K;
        // largest |Re|, |Im| of the row
        float m = 0.f;
        for (int q = lane; 4 * q < K; q += 32) {
            float4 a, b;
            load_quad<VEC>(x, 4 * q, K, a, b);
            m = fmaxf(m, fmaxf(amax4(a), amax4(b)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // 2^e m in [2^14, 2^15); e limited so that 2^e and 2^-e are normal floats
        int e = 0;
        if (m > 0.f && m <= 3.4e38f) {
            int k = 0;
            frexpf(m, &k);  // m < 2^k
            e = min(126, max(-126, 15 - k));
        }
        const float sc = ldexpf(1.0f, e);
        if (lane == 0) row_scale[row] = ldexpf(1.0f, -e);
        const long long chan = row / n_in;
        const int in = (int)(row - chan * n_in);
        // element offset of plane pl, in units of 4 halves (uint2)
        auto at = [&](int pl, int q) { return ((chan * NPL + pl) * n_in + in) * (long long)nq + q; };
        for (int q = lane; q < nq; q += 32) {
            float4 a, b;
            load_quad<VEC>(x, 4 * q, K, a, b);
            a = make_float4(a.x * sc, a.y * sc, a.z * sc, a.w * sc);
            b = make_float4(b.x * sc, b.y * sc, b.z * sc, b.w * sc);
            const __half2 r01 = __floats2half2_rn(a.x, a.z), r23 = __floats2half2_rn(b.x, b.z);
            const __half2 i01 = __floats2half2_rn(a.y, a.w), i23 = __floats2half2_rn(b.y, b.w);
            out[at(0, q)] = make_uint2(h2u(r01), h2u(r23));
            out[at(1, q)] = make_uint2(h2u(i01), h2u(i23));
            if constexpr (NPL == 4) {
                const float2 fr01 = __half22float2(r01), fr23 = __half22float2(r23);
                const float2 fi01 = __half22float2(i01), fi23 = __half22float2(i23);
                const __half2 lr01 = __floats2half2_rn(a.x - fr01.x, a.z - fr01.y);
                const __half2 lr23 = __floats2half2_rn(b.x - fr23.x, b.z - fr23.y);
                const __half2 li01 = __floats2half2_rn(a.y - fi01.x, a.w - fi01.y);
                const __half2 li23 = __floats2half2_rn(b.y - fi23.x, b.w - fi23.y);
                out[at(2, q)] = make_uint2(h2u(lr01), h2u(lr23));
                out[at(3, q)] = make_uint2(h2u(li01), h2u(li23));
            }
        }
    }
}

// The same conversion with the row held in registers: one CTA of 256 threads per
// (channel, input) row, CPT consecutive spectra per thread (CPT = 8 or 16, rows of up
// to 2048 or 4096 spectra), so the row is read from HBM once; the row maximum is a
// block reduction. Each thread writes 8 or 16 FP16 values (16-byte pieces) per plane.
template <int NPL, int CPT>
__global__ void __launch_bounds__(256) k_to_planar_row(const float2 *__restrict__ X, __half *__restrict__ out,
                                                       float *__restrict__ row_scale, int n_in, int K, int Kp) {
    __shared__ float red[8];
    const long long row = blockIdx.x;
    const float2 *x = X + row * K;
    const int s0 = threadIdx.x * CPT;
    float2 v[CPT];
    const bool vec = (K % 2) == 0;  // 16-byte aligned rows: pairs of spectra per load
#pragma unroll
    for (int e = 0; e < CPT; e += 2) {
        const int s = s0 + e;
        if (vec && s + 2 <= K) {
            const float4 q = __ldg(reinterpret_cast<const float4 *>(x + s));
            v[e] = make_float2(q.x, q.y);
            v[e + 1] = make_float2(q.z, q.w);
        } else {
            v[e] = s < K ? __ldg(x + s) : make_float2(0.f, 0.f);
            v[e + 1] = s + 1 < K ? __ldg(x + s + 1) : make_float2(0.f, 0.f);
        }
    }
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < CPT; ++e) m = fmaxf(m, fmaxf(fabsf(v[e].x), fabsf(v[e].y)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
    int e2 = 0;
    if (m > 0.f && m <= 3.4e38f) {
        int k = 0;
        frexpf(m, &k);
        e2 = min(126, max(-126, 15 - k));
    }
    const float sc = ldexpf(1.0f, e2);
    if (threadIdx.x == 0) row_scale[row] = ldexpf(1.0f, -e2);
    if (s0 >= Kp) return;
    const long long chan = row / n_in;
    const int in = (int)(row - chan * n_in);
    __half *base = out + ((chan * NPL) * n_in + in) * (long long)Kp + s0;
    const long long plane = (long long)n_in * Kp;
#pragma unroll
    for (int e = 0; e < CPT; e += 8) {
        if (s0 + e >= Kp) break;
        uint32_t hr[4], hi[4], lr[4], li[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 a = make_float2(v[e + 2 * q].x * sc, v[e + 2 * q].y * sc);
            const float2 b = make_float2(v[e + 2 * q + 1].x * sc, v[e + 2 * q + 1].y * sc);
            const __half2 r = __floats2half2_rn(a.x, b.x), i = __floats2half2_rn(a.y, b.y);
            hr[q] = h2u(r);
            hi[q] = h2u(i);
            if constexpr (NPL == 4) {
                const float2 fr = __half22float2(r), fi = __half22float2(i);
                lr[q] = h2u(__floats2half2_rn(a.x - fr.x, b.x - fr.y));
                li[q] = h2u(__floats2half2_rn(a.y - fi.x, b.y - fi.y));
            }
        }
        *reinterpret_cast<uint4 *>(base + e) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
        *reinterpret_cast<uint4 *>(base + plane + e) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if constexpr (NPL == 4) {
            *reinterpret_cast<uint4 *>(base + 2 * plane + e) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
            *reinterpret_cast<uint4 *>(base + 3 * plane + e) = make_uint4(li[0], li[1], li[2], li[3]);
        }
    }
}

template <int NPL>
void launch_np(bool vec, unsigned blocks, const float2 *X, uint2 *out, float *rsc, long long n_rows, int n_in, int K,
               int Kp, cudaStream_t st) {
    if (vec)
        k_to_planar<NPL, true><<<blocks, 32 * kWarps, 0, st>>>(X, out, rsc, n_rows, n_in, K, Kp);
    else
        k_to_planar<NPL, false><<<blocks, 32 * kWarps, 0, st>>>(X, out, rsc, n_rows, n_in, K, Kp);
}

// Complex int8 [chan][input][K] -> planar FP16 codes [chan][2][input][Kp] (the same
// integers, exact in FP16), zeros past K: one thread per 8 spectra of one row.
// x ^ 0x80 is the offset-binary code x + 128; under the high byte 0x64 it is the
// FP16 value 1024 + (x + 128), from which 1152 is subtracted exactly.
template <bool VEC>
__global__ void __launch_bounds__(256) k_i8_to_planar(const char2 *__restrict__ X, uint4 *__restrict__ out,
                                                      long long n_chunks, int n_in, int K, int Kp) {
    const int cpr = Kp / 8;  // 8-spectrum chunks per padded row
    const uint32_t k1152 = 0x64806480u;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_chunks;
         q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / cpr;
        const int s0 = 8 * (int)(q - row * cpr);
        const char2 *x = X + row * K;
        uint32_t w[4];
        if (VEC) {  // K % 8 == 0: rows and chunks are 16-byte aligned
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(x + s0));
            w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint32_t lo = 0, hi = 0;
                if (s0 + 2 * e < K) {
                    const char2 c = x[s0 + 2 * e];
                    lo = (uint32_t)(uint8_t)c.x | ((uint32_t)(uint8_t)c.y << 8);
                }
                if (s0 + 2 * e + 1 < K) {
                    const char2 c = x[s0 + 2 * e + 1];
                    hi = (uint32_t)(uint8_t)c.x | ((uint32_t)(uint8_t)c.y << 8);
                }
                w[e] = lo | (hi << 16);
            }
        }
        uint32_t re[4], im[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t u = w[e] ^ 0x80808080u;  // [re0 im0 re1 im1] + 128 each
            __half2 hr = __hsub2(__halves2half2(__ushort_as_half((unsigned short)(0x6400u | (u & 0xffu))),
                                                __ushort_as_half((unsigned short)(0x6400u | ((u >> 16) & 0xffu)))),
                                 *reinterpret_cast<const __half2 *>(&k1152));
            __half2 hi = __hsub2(__halves2half2(__ushort_as_half((unsigned short)(0x6400u | ((u >> 8) & 0xffu))),
                                                __ushort_as_half((unsigned short)(0x6400u | (u >> 24)))),
                                 *reinterpret_cast<const __half2 *>(&k1152));
            re[e] = h2u(hr);
            im[e] = h2u(hi);
        }
        // zero codes past K (the offset arithmetic above maps a zero byte pair to 0 already)
        const long long chan = row / n_in;
        const int in = (int)(row - chan * n_in);
        const long long o = ((chan * 2) * n_in + in) * (long long)cpr + s0 / 8;
        out[o] = make_uint4(re[0], re[1], re[2], re[3]);
        out[o + (long long)n_in * cpr] = make_uint4(im[0], im[1], im[2], im[3]);
    }
}

}  // namespace

int planar_kstride(int K) { return (K + 7) & ~7; }

corr_status launch_i8_to_planar(const Handle &h, const void *X, void *ws, cudaStream_t st) {
    const int K = h.n_spectra, Kp = planar_kstride(K);
    const long long n_chunks = (long long)h.n_chan * h.n_in * (Kp / 8);
    long long blocks = (n_chunks + 255) / 256;
    const long long cap = (long long)h.n_sm * 16;
    if (blocks > cap) blocks = cap;
    const bool vec = (K % 8) == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    if (vec)
        k_i8_to_planar<true><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const char2 *>(X), static_cast<uint4 *>(ws),
                                                               n_chunks, h.n_in, K, Kp);
    else
        k_i8_to_planar<false><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const char2 *>(X),
                                                                static_cast<uint4 *>(ws), n_chunks, h.n_in, K, Kp);
    return check_launch("k_i8_to_planar");
}

size_t planar_ws_bytes(const Handle &h, int npl) {
    return align16((size_t)h.n_chan * npl * h.n_in * planar_kstride(h.n_spectra) * 2) +
           sizeof(float) * (size_t)h.n_chan * h.n_in;
}

corr_status launch_to_planar(const Handle &h, const float2 *X, void *ws, int npl, cudaStream_t st) {
    const int K = h.n_spectra, Kp = planar_kstride(K);
    const long long n_rows = (long long)h.n_chan * h.n_in;
    float *rsc = planar_row_scale(h, ws, npl);
    long long blocks = (n_rows + kWarps - 1) / kWarps;
    const long long cap = (long long)h.n_sm * 16;
    if (blocks > cap) blocks = cap;
    // 16-byte loads need every row start 16-byte aligned: K even and an aligned buffer
    const bool vec = (K % 2) == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    uint2 *out = static_cast<uint2 *>(ws);
    if (Kp <= 4096 && n_rows <= 0x7fffffffLL && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
        // rows of up to 4096 spectra: held in registers, read once
        __half *o = static_cast<__half *>(ws);
        const unsigned nb = (unsigned)n_rows;
        if (npl == 2 && Kp <= 2048) k_to_planar_row<2, 8><<<nb, 256, 0, st>>>(X, o, rsc, h.n_in, K, Kp);
        else if (npl == 2) k_to_planar_row<2, 16><<<nb, 256, 0, st>>>(X, o, rsc, h.n_in, K, Kp);
        else if (Kp <= 2048) k_to_planar_row<4, 8><<<nb, 256, 0, st>>>(X, o, rsc, h.n_in, K, Kp);
        else k_to_planar_row<4, 16><<<nb, 256, 0, st>>>(X, o, rsc, h.n_in, K, Kp);
        return check_launch("k_to_planar_row");
    }
    if (npl == 2)
        launch_np<2>(vec, (unsigned)blocks, X, out, rsc, n_rows, h.n_in, K, Kp, st);
    else
        launch_np<4>(vec, (unsigned)blocks, X, out, rsc, n_rows, h.n_in, K, Kp, st);
    return check_launch("k_to_planar");
}

float *planar_row_scale(const Handle &h, void *ws, int npl) {
    return reinterpret_cast<float *>(static_cast<char *>(ws) +
                                     align16((size_t)h.n_chan * npl * h.n_in * planar_kstride(h.n_spectra) * 2));
}

}  // namespace corr
