// Complex float channelised data -> planar FP16 operands for the TMA X-engine.
//   plain (2 planes):  h = fp16(x) for Re and Im
//   hi/lo (4 planes):  h = fp16(x), l = fp16(x - h) for Re and Im, so that
//                      x = h + l to about 2^-22 relative and
//                      x_i conj(x_j) ~ h_i conj(h_j) + h_i conj(l_j) + l_i conj(h_j)
// (the l l term, ~2^-22 relative, is dropped). x - h is exact in FP32. Layout
// [chan][plane][input][spectrum], planes Re_h, Im_h (, Re_l, Im_l). One HBM pass:
// read 8 B, write 4 B (plain) or 8 B (hi/lo) per complex sample.
#include <cuda_fp16.h>

#include "internal.h"

namespace corr {
namespace {

template <int NPL>
__global__ void __launch_bounds__(256) k_to_planar(const float4 *__restrict__ X, uint2 *__restrict__ out,
                                                   long long n_quads, int n_in, int K) {
    // one thread: 4 consecutive spectra (2 x float4 = 4 complex) of one (channel, input) row
    const int qpr = K / 4;  // quads per row
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n_quads;
         q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / qpr;  // chan * n_in + input
        const int s4 = (int)(q - row * qpr);
        const long long chan = row / n_in;
        const int in = (int)(row - chan * n_in);
        const float4 a = __ldg(X + 2 * q), b = __ldg(X + 2 * q + 1);  // (re0 im0 re1 im1), (re2 im2 re3 im3)
        const __half2 r01 = __floats2half2_rn(a.x, a.z), r23 = __floats2half2_rn(b.x, b.z);
        const __half2 i01 = __floats2half2_rn(a.y, a.w), i23 = __floats2half2_rn(b.y, b.w);
        // element offset of plane p: ((chan * NPL + p) * n_in + in) * K + 4 * s4, in units of 4 halves (uint2)
        auto at = [&](int pl) { return ((chan * NPL + pl) * n_in + in) * (long long)(K / 4) + s4; };
        out[at(0)] = make_uint2(*reinterpret_cast<const uint32_t *>(&r01), *reinterpret_cast<const uint32_t *>(&r23));
        out[at(1)] = make_uint2(*reinterpret_cast<const uint32_t *>(&i01), *reinterpret_cast<const uint32_t *>(&i23));
        if constexpr (NPL == 4) {
            const float2 fr01 = __half22float2(r01), fr23 = __half22float2(r23);
            const float2 fi01 = __half22float2(i01), fi23 = __half22float2(i23);
            const __half2 lr01 = __floats2half2_rn(a.x - fr01.x, a.z - fr01.y);
            const __half2 lr23 = __floats2half2_rn(b.x - fr23.x, b.z - fr23.y);
            const __half2 li01 = __floats2half2_rn(a.y - fi01.x, a.w - fi01.y);
            const __half2 li23 = __floats2half2_rn(b.y - fi23.x, b.w - fi23.y);
            out[at(2)] = make_uint2(*reinterpret_cast<const uint32_t *>(&lr01), *reinterpret_cast<const uint32_t *>(&lr23));
            out[at(3)] = make_uint2(*reinterpret_cast<const uint32_t *>(&li01), *reinterpret_cast<const uint32_t *>(&li23));
        }
    }
}

}  // namespace

corr_status launch_to_planar(const Handle &h, const float2 *X, void *out, int npl, cudaStream_t st) {
    if ((h.n_spectra % 4) != 0) return CORR_EUNSUPPORTED;
    const long long n_quads = (long long)h.n_chan * h.n_in * (h.n_spectra / 4);
    long long blocks = (n_quads + 255) / 256;
    const long long cap = (long long)h.n_sm * 16;
    if (blocks > cap) blocks = cap;
    if (npl == 2)
        k_to_planar<2><<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(X),
                                                         static_cast<uint2 *>(out), n_quads, h.n_in, h.n_spectra);
    else
        k_to_planar<4><<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const float4 *>(X),
                                                         static_cast<uint2 *>(out), n_quads, h.n_in, h.n_spectra);
    return check_launch("k_to_planar");
}

}  // namespace corr
