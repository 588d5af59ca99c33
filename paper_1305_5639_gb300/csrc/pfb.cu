// Polyphase filter-bank front end: the FIR pass. For spectrum a of input i it forms
//     y_a[n] = sum_{p < P} h[p][n] s'_i[(a + p) N + n],    n < N,
// with s'_i[t] = s_i[t + D_i] (the integer delay advance, D_i = 0 without delays)
// and zero wherever t + D_i is not a recorded sample, and writes the frames as
// complex FP32 [n_in][K][N] for the F-engine's FFT (which then applies the
// fractional delay phase). One thread per (input, 4 consecutive positions, run of
// 16 spectra): consecutive threads take consecutive positions, so loads and stores
// are coalesced and vectorised, and the P - 1 frames a spectrum shares with the
// previous one come from L1 (this kernel uses no shared memory, so L1 keeps its
// full size). HBM: the raw samples once, 8 bytes written per sample.
#include "internal.h"

namespace corr {
namespace {

constexpr int kFirThreads = 256;
constexpr int kFirRun = 16;  // spectra per thread
constexpr int kFirVec = 4;   // consecutive positions per thread (one 8- or 32-byte load per tap)

template <bool I8>
__global__ void __launch_bounds__(kFirThreads) k_pfb_fir(const void *__restrict__ volt, const float *__restrict__ win,
                                                         int P, const int *__restrict__ dint,
                                                         float2 *__restrict__ y, int N, int K, int i0) {
    const int i = i0 + blockIdx.y;
    const long long g = (long long)blockIdx.x * kFirThreads + threadIdx.x;
    const int nq = N / kFirVec;  // position quads per frame
    const int n_runs = (K + kFirRun - 1) / kFirRun;
    if (g >= (long long)nq * n_runs) return;
    const int n = (int)(g % nq) * kFirVec, run = (int)(g / nq);
    const long long n_rec = (long long)K * N;
    const long long D = dint ? (long long)__ldg(dint + i) : 0;
    const long long base = (long long)i * n_rec;
    // with a delay the quad may straddle 4-sample boundaries: element loads then
    const bool vec = (D % kFirVec) == 0;
    const int a0 = run * kFirRun, a1 = min(K, a0 + kFirRun);
    for (int a = a0; a < a1; ++a) {
        float2 acc[kFirVec];
#pragma unroll
        for (int e = 0; e < kFirVec; ++e) acc[e] = make_float2(0.f, 0.f);
        for (int p = 0; p < P; ++p) {
            const long long t = (long long)(a + p) * N + n + D;  // first sample of the quad
            if (t + kFirVec <= 0 || t >= n_rec) continue;
            float2 x[kFirVec];
            if (vec && t >= 0 && t + kFirVec <= n_rec) {
                if constexpr (I8) {
                    const int2 w = __ldg(reinterpret_cast<const int2 *>(reinterpret_cast<const char2 *>(volt) + base + t));
                    const uint32_t u[2] = {(uint32_t)w.x, (uint32_t)w.y};
#pragma unroll
                    for (int e = 0; e < kFirVec; ++e) {
                        const uint32_t b = u[e >> 1] >> (16 * (e & 1));
                        x[e] = make_float2((float)(int8_t)(b & 0xff), (float)(int8_t)((b >> 8) & 0xff));
                    }
                } else {
                    const float4 *src = reinterpret_cast<const float4 *>(reinterpret_cast<const float2 *>(volt) + base + t);
                    const float4 q0 = __ldg(src), q1 = __ldg(src + 1);
                    x[0] = make_float2(q0.x, q0.y), x[1] = make_float2(q0.z, q0.w);
                    x[2] = make_float2(q1.x, q1.y), x[3] = make_float2(q1.z, q1.w);
                }
            } else {
#pragma unroll
                for (int e = 0; e < kFirVec; ++e) {
                    const long long te = t + e;
                    x[e] = make_float2(0.f, 0.f);
                    if (te >= 0 && te < n_rec) {
                        if constexpr (I8) {
                            const char2 c = __ldg(reinterpret_cast<const char2 *>(volt) + base + te);
                            x[e] = make_float2((float)c.x, (float)c.y);
                        } else {
                            x[e] = __ldg(reinterpret_cast<const float2 *>(volt) + base + te);
                        }
                    }
                }
            }
            const float4 w = __ldg(reinterpret_cast<const float4 *>(win + (size_t)p * N + n));
            const float wv[kFirVec] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < kFirVec; ++e) {
                acc[e].x = fmaf(wv[e], x[e].x, acc[e].x);
                acc[e].y = fmaf(wv[e], x[e].y, acc[e].y);
            }
        }
        float4 *dst = reinterpret_cast<float4 *>(y + base + (long long)a * N + n);
        dst[0] = make_float4(acc[0].x, acc[0].y, acc[1].x, acc[1].y);
        dst[1] = make_float4(acc[2].x, acc[2].y, acc[3].x, acc[3].y);
    }
}

}  // namespace

corr_status launch_pfb_fir(const Handle &h, const void *volt, int i0, int n_run, cudaStream_t st) {
    if (n_run <= 0) return CORR_OK;
    // aligned vector loads: 16-byte aligned inputs (checked by the API) and N % 4 == 0
    const long long threads = (long long)(h.n_chan / kFirVec) * ((h.n_spectra + kFirRun - 1) / kFirRun);
    const long long blocks = (threads + kFirThreads - 1) / kFirThreads;
    if (blocks > 0x7fffffffLL || n_run > 65535) return CORR_EUNSUPPORTED;
    dim3 grid((unsigned)blocks, (unsigned)n_run);
    if (h.precision == CORR_PREC_INT8)
        k_pfb_fir<true><<<grid, kFirThreads, 0, st>>>(volt, h.pfb_win, h.pfb_taps, h.dly_int,
                                                      static_cast<float2 *>(h.pfb_y), h.n_chan, h.n_spectra, i0);
    else
        k_pfb_fir<false><<<grid, kFirThreads, 0, st>>>(volt, h.pfb_win, h.pfb_taps, h.dly_int,
                                                       static_cast<float2 *>(h.pfb_y), h.n_chan, h.n_spectra, i0);
    return check_launch("k_pfb_fir");
}

}  // namespace corr
