// F-engine: per-input channelisation by an unnormalised forward DFT (Eq. 1,
// Section 2), 8-bit re-packing of the spectra and corner turn to channel-major
// order, in one pass.
//
// Each N = T1 x T2 point FFT is computed by a group of max(T1, T2) threads in two
// register passes (four-step / Cooley-Tukey split n = t + T2 m, k = k1 + T1 k2):
//   pass 1: thread t < T2 holds x[t + T2 m], m < T1, and computes the T1-point DFT
//           over m; the result is multiplied by W_N^(t k1) (twiddle table copied
//           to shared memory per CTA)
//   exchange through shared memory (padded rows, conflict-free)
//   pass 2: thread k1 < T1 holds Y[t][k1], t < T2, and computes the T2-point DFT
//           over t, giving X[k1 + T1 k2].
// Square lengths (16, 64, 256, 1024) keep every thread busy in both passes; the
// others (128, 512, 2048, 4096: T2 = 2 T1 or T1 = T2 = 64) leave the threads past
// the shorter dimension idle in one pass.
// A CTA handles one input and SB consecutive spectra; the outputs are staged in
// shared memory as [channel][spectrum] so that every (channel, input) row segment
// of SB spectra is written to global memory contiguously (the corner turn). Raw
// int8 frames of the plain front end arrive by asynchronous copies into the FFT's
// exchange buffer while the previous frame's pass 2 runs, and enter pass 1 scaled by
// 256 on an offset that the first butterflies cancel (i8_to_f2_scaled).
//
// This header holds the kernel template; the per-feature translation units
// (fengine_plain.cu, fengine_delay.cu) instantiate it, so that the instantiations
// compile in parallel, and fengine.cu holds the host entry points.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda_fp16.h>

#include "fft_common.cuh"
#include "internal.h"
#include "requant.cuh"

namespace corr {

// Shape and twiddle table of one F-engine launch.
struct FShape {
    int n_in, n_chan, n_spectra;
    bool i8;
    const float2 *tw;  // [k1][t] table for n_chan = T1 x T2
    int i0 = 0, n_run = -1;  // inputs [i0, i0 + n_run) of the n_in (n_run < 0: all)
    const int *dint = nullptr;     // per-input integer advance (delay compensation), or null
    const float2 *dph = nullptr;   // per-input phase tables [n_in][T1 + T2]: c[k1], then d[k2]
};

namespace {


constexpr int kThreads = 256;

enum Mode { kFloatOut = 0, kRequant = 1, kPower = 2, kRequantPlanar = 3 };

template <int N, bool I8, int MODE>
struct FCfg {
    static constexpr int T2 = fengine_t2(N);  // pass-1 threads = pass-2 DFT length
    static constexpr int T1 = N / T2;         // pass-1 DFT length = pass-2 threads
    static_assert(T2 > 0 && T1 * T2 == N && T1 <= T2 && T2 <= 64, "unsupported F-engine length");
    static constexpr int TG = T2;             // threads per FFT group
    static constexpr int G = kThreads / TG;   // FFTs in flight per CTA
    // Exchange buffer of one FFT: T1 rows of EXS floats; row k1 receives Y[0..T2-1][k1]
    // (one column per writing thread) and is read back as float4. EXS and the per-FFT
    // stride GS keep both the scalar writes and the float4 reads free of bank conflicts:
    // 4 EXS / 4 odd per quarter warp, and GS = TG (mod 32) so that the FFTs sharing a
    // warp write to disjoint banks.
    static constexpr int EXS = T2 == 4 ? 8 : T2 + 4;
    static constexpr int GS = T1 * EXS + (TG >= 32 ? 0 : TG);
    static constexpr bool RQ = MODE == kRequant || MODE == kRequantPlanar;
    // spectra per CTA: the re-packing modes take 32 up to N = 1024 (64-byte row
    // segments of the planar FP16 planes, 2 CTAs/SM at N = 1024), fewer for longer
    // transforms so that the staging rows stay at 64 KB
    static constexpr int SB = MODE == kFloatOut ? (N <= 1024 ? 8 : 8192 / N) : (RQ ? (N <= 1024 ? 32 : 32768 / N) : 16);
    // staging row stride in 32-bit words. The re-packing modes stage one 16-bit code
    // pair per (channel k, spectrum s): a row of SB / 2 words whose word index is
    // XOR-swizzled with (k >> SW) & (ROWW - 1), SW = log2(32 / ROWW), so that the
    // 16-bit writes of one warp (32 consecutive rows) and the 4-word row reads of the
    // copy-out are free of bank conflicts. The FP32 mode stages float2 values in
    // padded rows.
    static constexpr int ROWW = RQ ? SB / 2 : (MODE == kFloatOut ? 2 * SB + 2 : 0);
    static constexpr int SW = RQ ? ilog2(32 / ROWW) : 0;
    static_assert(!RQ || (ROWW >= 4 && ROWW <= 16), "swizzle assumes 4..16-word rows");
    static constexpr size_t ex_bytes = sizeof(float) * (size_t)G * GS;
    static constexpr size_t pw_bytes = MODE == kPower ? sizeof(float) * N : 0;
    static constexpr size_t tw_bytes = sizeof(float2) * (size_t)N;  // twiddle table copy
    static constexpr size_t dl_bytes = sizeof(float2) * 64;         // delay phases d[k2] (T2 <= 64)
    static constexpr size_t st_bytes = sizeof(uint32_t) * (size_t)N * ROWW;
    static constexpr size_t smem = ex_bytes + pw_bytes + tw_bytes + dl_bytes + st_bytes;
    static_assert(smem <= 232448, "shared memory");
};

// complex int8 sample (16 bits: re in the low byte) -> float2, exactly:
// (0x4B400000 | (x + 128)) is the float 12582912 + x + 128.
__device__ __forceinline__ float2 i8_to_f2(uint32_t w) {
    const uint32_t u = w ^ 0x8080u;
    return f2_sub(make_float2(__uint_as_float(__byte_perm(u, 0x4B400000u, 0x7650)),
                              __uint_as_float(__byte_perm(u, 0x4B400000u, 0x7651))),
                  make_float2(kMagic + 128.0f, kMagic + 128.0f));
}

// complex int8 sample x (16 bits: re in the low byte) -> float2 (c + 256 re, c + 256 im)
// with the constant c = 2^23 + 2^15, exactly: the float with bits 0x4B00 (x + 128) 00
// is 2^23 + 256 (x + 128). The offset needs no subtraction here: the first radix-2
// stage's differences cancel it exactly, and along the all-sums path (DFT bin 0 of
// pass 1) every partial sum j c + 256 s stays exact (a multiple of 256 below 2^29,
// where the spacing of floats is at most 32), so that bin is corrected once per FFT
// (kOffsetFix). The factor 256 leaves every rounding unchanged (a power of two); it
// is divided out by the inter-pass twiddles, stored divided by 256.
__device__ __forceinline__ float2 i8_to_f2_scaled(uint32_t w) {
    const uint32_t u = w ^ 0x8080u;
    return make_float2(__uint_as_float(__byte_perm(u, 0x4B000000u, 0x7404)),
                       __uint_as_float(__byte_perm(u, 0x4B000000u, 0x7414)));
}
constexpr float kI8Scale = 256.0f;
constexpr float kI8OffsetOverScale = 32896.0f;  // (2^23 + 2^15) / 256

// pass-1 bin 0 of T scaled samples (T c + 256 sum x, exact below 2^31: every partial
// sum is a multiple of 256) -> sum x, exactly
template <int T>
__device__ __forceinline__ float2 kOffsetFix(float2 v) {
    constexpr float k = -(float)T * kI8OffsetOverScale;
    return f2_fma(v, make_float2(1.0f / kI8Scale, 1.0f / kI8Scale), make_float2(k, k));
}

// 16-byte global -> shared copy that bypasses the registers (cp.async, L2 only)
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Front-end features of one F-engine instantiation: none, or delay compensation
// (an integer advance of the frames and / or the per-channel fractional phase).
enum Feat { kPlain = 0, kDelay = 1 };

template <int N, bool I8, int MODE, int FEAT>
__global__ void __launch_bounds__(kThreads, (N >= 2048 || (MODE == kPower && N >= 512)) ? 1 : (N >= 512 ? 2 : 3)) k_fengine(const void *__restrict__ volt,
                                                      const float *__restrict__ scale,
                                                      void *__restrict__ out,
                                                      double *__restrict__ power, int n_in, int K,
                                                      const float2 *__restrict__ tw_glob, int i0, int vec_out,
                                                      const int *__restrict__ dint,
                                                      const float2 *__restrict__ dph, int async_raw) {
    using C = FCfg<N, I8, MODE>;
    constexpr int T1 = C::T1, T2 = C::T2, TG = C::TG, G = C::G, EXS = C::EXS, SB = C::SB, ROWW = C::ROWW;
    constexpr int TV = T1 > T2 ? T1 : T2;  // register values per thread
    // square 32- or 64-point passes read the exchange into float arrays and do pass 2's
    // first stage in scalar arithmetic (no register moves into the (re, im) pairs); the
    // smaller lengths keep the in-place reads, which fit their register budgets
    constexpr bool kScalarStage = T1 == T2 && T2 >= 32;
    constexpr bool DLY = FEAT == kDelay;  // delay code compiled in
    // int8 samples enter the plain FFT scaled by 256 on an offset (i8_to_f2_scaled); the
    // delay instantiation converts them exactly (measured faster there)
    constexpr bool SCALED = I8 && !DLY;
    // the integer advance and the phase are separate: the filter-bank path applies the
    // advance in its FIR pass and only the phase here
    const bool has_shift = DLY && dint != nullptr, has_dly = DLY && dph != nullptr;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *ex = reinterpret_cast<float *>(smem_raw);                                 // [G][T1][EXS]
    float *scs = reinterpret_cast<float *>(smem_raw + C::ex_bytes);                  // [N] (power)
    float2 *tws = reinterpret_cast<float2 *>(smem_raw + C::ex_bytes + C::pw_bytes);  // [k1][t] twiddles
    float2 *dsm = reinterpret_cast<float2 *>(smem_raw + C::ex_bytes + C::pw_bytes + C::tw_bytes);  // [k2] phases
    uint32_t *stg = reinterpret_cast<uint32_t *>(smem_raw + C::ex_bytes + C::pw_bytes + C::tw_bytes +
                                                 C::dl_bytes);  // staging
    // 16-bit slot of code (k, s) in the swizzled staging rows
    auto slot = [](int k, int s) {
        return k * (2 * ROWW) + 2 * ((s >> 1) ^ ((k >> C::SW) & (ROWW - 1))) + (s & 1);
    };
    // the threads of one FFT group meet: a warp (or part of one), or the whole CTA
    auto group_sync = [] {
        if constexpr (TG <= 32) __syncwarp(); else __syncthreads();
    };

    const int i = i0 + blockIdx.y;
    const int a0 = blockIdx.x * SB;
    // Raw int8 frames without delays are copied asynchronously into the FFT's exchange
    // buffer (free between exchanges): the copy for the next frame is issued after the
    // current frame's exchange and lands while its pass 2 and re-packing run. Each of
    // the TG threads moves N / (8 TG) 16-byte pieces of the 2 N-byte frame.
    constexpr bool kAsync = I8 && !DLY && N / (8 * TG) >= 1;
    static_assert(!kAsync || sizeof(float) * C::GS >= 2 * N, "exchange buffer holds one raw frame");
    const bool use_async = kAsync && async_raw;
    // copy of frame s_ of this CTA into the exchange buffer of FFT slot s_ % G
    auto issue_raw = [&](int s_) {
        const int a_ = a0 + s_, t_ = threadIdx.x % TG;
        if (s_ < SB && a_ < K) {
            const char *src = reinterpret_cast<const char *>(volt) + ((size_t)i * K + a_) * (size_t)N * 2;
            char *dst = reinterpret_cast<char *>(ex + (size_t)(s_ % G) * C::GS);
#pragma unroll
            for (int c = 0; c < N / (8 * TG); ++c) cp_async16(dst + (c * TG + t_) * 16, src + (c * TG + t_) * 16);
        }
        cp_async_commit();
    };
    if (use_async) issue_raw(threadIdx.x / TG);
    // Delay compensation: the frames are read D samples later in input i's stream
    // (samples outside the record are zero) and channel k = k1 + T1 k2 is multiplied by
    // c[k1] d[k2] = exp(+j 2 pi k f / N): c is folded into the inter-pass twiddles
    // (it is common to thread k1's pass-2 DFT), d applied to the outputs.
    const long long n_rec = (long long)K * N;  // samples per input
    const int D = has_shift ? __ldg(dint + i) : 0;
    {
        // Warm L2 with this CTA's raw block (SB consecutive spectra of input i, one
        // contiguous range): the loads of the later spectra then hit L2 instead of HBM.
        constexpr int BPS = I8 ? 2 : 8;  // bytes per complex sample
        const long long lo = max(0LL, (long long)a0 * N + D);
        const long long hi = min(n_rec, (long long)min(K, a0 + SB) * N + D);
        if (hi > lo) {
            const char *blk = reinterpret_cast<const char *>(volt) + ((size_t)i * n_rec + lo) * BPS;
            const int lines = (int)(((hi - lo) * BPS + 127) / 128);
            for (int l = threadIdx.x; l < lines; l += kThreads)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(blk + (size_t)l * 128));
        }
    }
    // per-CTA copy of the twiddle table (shared-memory loads in the FFT loop; measured
    // faster than L1 lookups, while the channel scales are faster from L1)
    for (int m = threadIdx.x; m < N; m += kThreads) {
        float2 w = __ldg(tw_glob + m);
        if (DLY && has_dly) {
            w = cmul(w, __ldg(dph + (size_t)i * (T1 + T2) + m / T2));  // table [k1][t]: c[k1]
            if (m < T2) dsm[m] = __ldg(dph + (size_t)i * (T1 + T2) + T1 + m);
        }
        if constexpr (SCALED) w = make_float2(w.x * (1.0f / kI8Scale), w.y * (1.0f / kI8Scale));
        tws[m] = w;
        if constexpr (MODE == kPower) scs[m] = 0.0f;
    }
    __syncthreads();

    const int g = threadIdx.x / TG;
    const int t = threadIdx.x % TG;
    // pass 1 uses threads t < T2 (the columns), pass 2 threads k1 = t < T1 (the rows)
    const bool act1 = T2 == TG || t < T2, act2 = T1 == TG || t < T1;
    float *exg = ex + (size_t)g * C::GS;
    const float4 *exrow = reinterpret_cast<const float4 *>(exg + (act2 ? t : 0) * EXS);
    float pw[T2];
    if constexpr (MODE == kPower) {
#pragma unroll
        for (int q = 0; q < T2; ++q) pw[q] = 0.0f;
    }

    for (int s0 = 0; s0 < SB; s0 += G) {
        const int s = s0 + g;
        const int a = a0 + s;
        const bool valid = (s < SB) && (a < K);
        const bool valid1 = valid && act1;
        float2 v[TV];
        // ---- pass 1: thread t takes x[t + T2 m]
        // sample offset of this frame in input i's stream (shifted by D with delays)
        const long long off = (long long)(valid ? a : 0) * N + D;
        const long long base = (long long)i * n_rec + off + t;
        // with delays, frames that reach outside the record take the checked loads
        const bool inside = !DLY || (off >= 0 && off + N <= n_rec);
        if constexpr (I8) {
            const unsigned short *src = reinterpret_cast<const unsigned short *>(volt) + base;
            if (use_async) {
                cp_async_wait_all();
                group_sync();  // every thread's pieces of the frame have landed
                const unsigned short *raw = reinterpret_cast<const unsigned short *>(exg) + t;
#pragma unroll
                for (int m = 0; m < T1; ++m) v[m] = i8_to_f2_scaled(valid1 ? (uint32_t)raw[T2 * m] : 0u);
                group_sync();  // read before the exchange overwrites the buffer
            } else if (inside) {
#pragma unroll
                for (int m = 0; m < T1; ++m) {
                    const uint32_t w = valid1 ? (uint32_t)__ldg(src + (size_t)T2 * m) : 0u;
                    v[m] = SCALED ? i8_to_f2_scaled(w) : i8_to_f2(w);
                }
            } else {
#pragma unroll
                for (int m = 0; m < T1; ++m) {
                    const long long n = off + t + T2 * m;
                    const uint32_t w = (valid1 && n >= 0 && n < n_rec) ? (uint32_t)__ldg(src + (long long)T2 * m) : 0u;
                    v[m] = SCALED ? i8_to_f2_scaled(w) : i8_to_f2(w);
                }
            }
        } else {
            const float2 *src = reinterpret_cast<const float2 *>(volt) + base;
            if (inside) {
#pragma unroll
                for (int m = 0; m < T1; ++m) v[m] = valid1 ? __ldg(src + (size_t)T2 * m) : make_float2(0.f, 0.f);
            } else {
#pragma unroll
                for (int m = 0; m < T1; ++m) {
                    const long long n = off + t + T2 * m;
                    v[m] = (valid1 && n >= 0 && n < n_rec) ? __ldg(src + (long long)T2 * m) : make_float2(0.f, 0.f);
                }
            }
        }
        fft_dif<T1>(v);  // v[bitrev(k1)] = Y[t][k1] (x 256, bin 0 offset, for int8 input)
        if constexpr (SCALED) v[0] = kOffsetFix<T1>(v[0]);
        sfor<0, T1>([&](auto K1) {
            constexpr int k1 = decltype(K1)::value;
            // twiddle W_N^(t k1), table laid out [k1][t]
            if constexpr (k1 != 0)
                if (act1) v[bitrev(k1, ilog2(T1))] = cmul(v[bitrev(k1, ilog2(T1))], tws[k1 * T2 + t]);
        });
        // ---- exchange (Re, then Im; the other half stays in place) and pass 2:
        // thread t now plays k1 = t and takes Y[tt][k1], tt < T2
        if (act1)
            sfor<0, T1>([&](auto K1) {
                constexpr int k1 = decltype(K1)::value;
                exg[k1 * EXS + t] = v[bitrev(k1, ilog2(T1))].x;
            });
        group_sync();
        if constexpr (kScalarStage) {
            // the rows are read into plain float arrays (a 16-byte load fills four
            // consecutive registers, which the (re, im) register pairs of v cannot offer)
            float rin[T2], iin[T2];
            if (act2) {
#pragma unroll
                for (int j = 0; j < T2 / 4; ++j) {
                    const float4 r = exrow[j];
                    rin[4 * j] = r.x, rin[4 * j + 1] = r.y, rin[4 * j + 2] = r.z, rin[4 * j + 3] = r.w;
                }
            }
            group_sync();
            if (act1)
                sfor<0, T1>([&](auto K1) {
                    constexpr int k1 = decltype(K1)::value;
                    exg[k1 * EXS + t] = v[bitrev(k1, ilog2(T1))].y;
                });
            group_sync();
            if (act2) {
#pragma unroll
                for (int j = 0; j < T2 / 4; ++j) {
                    const float4 r = exrow[j];
                    iin[4 * j] = r.x, iin[4 * j + 1] = r.y, iin[4 * j + 2] = r.z, iin[4 * j + 3] = r.w;
                }
            }
            group_sync();
            if (use_async && s0 + G < SB) issue_raw(s0 + G + g);  // next frame into the free buffer
            // pass 2: its first radix-2 stage in scalar arithmetic, from the float arrays
            // into the (re, im) pairs, then the remaining stages on the pairs
            sfor<0, T2 / 2>([&](auto J) {
                constexpr int a = decltype(J)::value, b = a + T2 / 2;
                const float ar = rin[a], ai = iin[a], br = rin[b], bi = iin[b];
                v[a] = make_float2(ar + br, ai + bi);
                if constexpr (4 * a == T2)
                    v[b] = make_float2(ai - bi, br - ar);  // (x - y)(-j)
                else
                    v[b] = mul_w<a, T2>(make_float2(ar - br, ai - bi));
            });
            fft_dif<T2, TV, 1>(v);  // v[bitrev(k2)] = X[t + T1 k2]
        } else {
            if (act2) {
#pragma unroll
                for (int j = 0; j < T2 / 4; ++j) {
                    const float4 r = exrow[j];
                    v[4 * j].x = r.x, v[4 * j + 1].x = r.y, v[4 * j + 2].x = r.z, v[4 * j + 3].x = r.w;
                }
            }
            group_sync();
            if (act1)
                sfor<0, T1>([&](auto K1) {
                    constexpr int k1 = decltype(K1)::value;
                    exg[k1 * EXS + t] = v[bitrev(k1, ilog2(T1))].y;
                });
            group_sync();
            if (act2) {
#pragma unroll
                for (int j = 0; j < T2 / 4; ++j) {
                    const float4 r = exrow[j];
                    v[4 * j].y = r.x, v[4 * j + 1].y = r.y, v[4 * j + 2].y = r.z, v[4 * j + 3].y = r.w;
                }
            }
            group_sync();
            if (use_async && s0 + G < SB) issue_raw(s0 + G + g);  // next frame into the free buffer
            fft_dif<T2>(v);  // v[bitrev(k2)] = X[t + T1 k2]
        }
        if (valid && act2) {
            sfor<0, T2>([&](auto K2) {
                constexpr int k2 = decltype(K2)::value;
                const int k = t + T1 * k2;
                float2 x = v[bitrev(k2, ilog2(T2))];
                if constexpr (DLY && k2 != 0) {
                    if (has_dly) x = cmul(x, dsm[k2]);  // delay phase exp(+j 2 pi T1 k2 f / N)
                }
                if constexpr (MODE == kRequant || MODE == kRequantPlanar) {
                    const uint32_t q = pack_q<MODE == kRequantPlanar>(x, __ldg(scale + k));
                    reinterpret_cast<uint16_t *>(stg)[slot(k, s)] = (uint16_t)q;
                } else if constexpr (MODE == kFloatOut) {
                    reinterpret_cast<float2 *>(stg)[(size_t)k * (ROWW / 2) + s] = x;
                } else {
                    pw[k2] += x.x * x.x + x.y * x.y;
                }
            });
        }
    }

    if constexpr (MODE != kPower) {
        __syncthreads();
        // ---- corner turn: row (k, i) gets spectra a0 .. a0 + nv - 1
        const int nv = min(SB, K - a0);
        if constexpr (MODE == kRequantPlanar || MODE == kRequant) {
            uint16_t *dst = reinterpret_cast<uint16_t *>(out);
            const uint16_t *sh = reinterpret_cast<const uint16_t *>(stg);
            // planar FP16 layout [k][plane][i][a]; int8 layout [k][i][a] (complex int8)
            constexpr int PL = MODE == kRequantPlanar ? 2 : 1;
            if (nv == SB && vec_out) {
                // each thread moves 8 spectra of one channel row: 4 staged words
                // (the code pairs of 2 spectra each) -> one 16-byte store per plane
                constexpr int CPR = SB / 8;          // 8-spectrum chunks per row
                constexpr int RPI = kThreads / CPR;  // rows per iteration
                const int q = threadIdx.x % CPR;
                int k = threadIdx.x / CPR;
                // physical words of logical words 4q .. 4q + 3 in row k; the swizzle
                // (k >> SW) & (ROWW - 1) is the same for k + RPI
                static_assert((RPI >> C::SW) % ROWW == 0 || RPI >= N, "");
                const int h = (k >> C::SW) & (ROWW - 1);
                const int o0 = (4 * q) ^ h, o1 = (4 * q + 1) ^ h, o2 = (4 * q + 2) ^ h, o3 = (4 * q + 3) ^ h;
                const uint32_t *src = stg + (size_t)k * ROWW;
                uint4 *d = reinterpret_cast<uint4 *>(dst + ((size_t)(PL * k) * n_in + i) * K + a0 + 8 * q);
                const size_t dstep = (size_t)PL * RPI * n_in * K / 8, dplane = (size_t)n_in * K / 8;
                for (; k < N; k += RPI, src += RPI * ROWW, d += dstep) {
                    const uint32_t w0 = src[o0], w1 = src[o1], w2 = src[o2], w3 = src[o3];
                    if constexpr (MODE == kRequantPlanar) {
                        uint4 re, im;
                        ob_codes_to_f16_planes(w0, re.x, im.x);
                        ob_codes_to_f16_planes(w1, re.y, im.y);
                        ob_codes_to_f16_planes(w2, re.z, im.z);
                        ob_codes_to_f16_planes(w3, re.w, im.w);
                        d[0] = re;
                        d[dplane] = im;
                    } else {
                        d[0] = make_uint4(w0, w1, w2, w3);
                    }
                }
            } else {
                for (int e = threadIdx.x; e < N * SB; e += kThreads) {
                    const int k = e / SB, c = e % SB;
                    if (c < nv) {
                        const uint16_t code = sh[slot(k, c)];
                        uint16_t *row0 = dst + ((size_t)(PL * k) * n_in + i) * K + a0;
                        if constexpr (MODE == kRequantPlanar) {
                            uint32_t re, im;
                            ob_codes_to_f16_planes((uint32_t)code, re, im);
                            row0[c] = (uint16_t)(re & 0xffffu);
                            row0[(size_t)n_in * K + c] = (uint16_t)(im & 0xffffu);
                        } else {
                            row0[c] = code;
                        }
                    }
                }
            }
        } else {
            float2 *dst = reinterpret_cast<float2 *>(out);
            const float2 *sh = reinterpret_cast<const float2 *>(stg);
            for (int e = threadIdx.x; e < N * SB; e += kThreads) {
                int k = e / SB, c = e % SB;
                if (c < nv) dst[((size_t)k * n_in + i) * K + a0 + c] = sh[(size_t)k * (ROWW / 2) + c];
            }
        }
    }

    if constexpr (MODE == kPower) {
        if (act2)
            sfor<0, T2>([&](auto K2) {
                constexpr int k2 = decltype(K2)::value;
                atomicAdd(&scs[t + T1 * k2], pw[k2]);
            });
        __syncthreads();
        for (int m = threadIdx.x; m < N; m += kThreads) atomicAdd(&power[m], (double)scs[m]);
    }
}

template <int N, bool I8, int MODE, int FEAT>
corr_status launch_one_(const FShape &f, const void *volt, const float *scale, void *out, double *power,
                       cudaStream_t st) {
    using C = FCfg<N, I8, MODE>;
    auto kern = k_fengine<N, I8, MODE, FEAT>;
    CORR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem));
    // 16-byte row stores need 16-byte aligned rows: an aligned buffer and 8 | n_spectra
    const int vec_out = (reinterpret_cast<uintptr_t>(out) % 16 == 0) && (f.n_spectra % 8 == 0);
    // blockIdx.x (the spectra block) varies fastest, so the CTAs resident at one time
    // write neighbouring segments of the same output rows
    dim3 grid((f.n_spectra + C::SB - 1) / C::SB, f.n_run < 0 ? f.n_in : f.n_run);
    // asynchronous raw copies need 16-byte aligned frames (2 N bytes each, N >= 64); the
    // public entry points only accept 16-byte aligned voltages, so this is a safeguard
    const int async_raw = reinterpret_cast<uintptr_t>(volt) % 16 == 0;
    kern<<<grid, kThreads, C::smem, st>>>(volt, scale, out, power, f.n_in, f.n_spectra, f.tw, f.i0, vec_out,
                                          f.dint, f.dph, async_raw);
    return check_launch("k_fengine");
}

template <int MODE, int FEAT>
corr_status launch_mode(const FShape &f, const void *volt, const float *scale, void *out, double *power,
                        cudaStream_t st) {
#define CORR_F_CASE(NN)                                                                      \
    case NN:                                                                                 \
        return f.i8 ? launch_one_<NN, true, MODE, FEAT>(f, volt, scale, out, power, st)      \
                    : launch_one_<NN, false, MODE, FEAT>(f, volt, scale, out, power, st);
    switch (f.n_chan) {
        CORR_F_CASE(16)
        CORR_F_CASE(64)
        CORR_F_CASE(128)
        CORR_F_CASE(256)
        CORR_F_CASE(512)
        CORR_F_CASE(1024)
        CORR_F_CASE(2048)
        CORR_F_CASE(4096)
        default: return CORR_EUNSUPPORTED;
    }
#undef CORR_F_CASE
}

// Every (mode, n_chan, input type) of one front-end feature.
template <int FEAT>
corr_status launch_feature(int mode, const FShape &f, const void *volt, const float *scale, void *out,
                           double *power, cudaStream_t st) {
    switch (mode) {
        case kFloatOut: return launch_mode<kFloatOut, FEAT>(f, volt, scale, out, power, st);
        case kRequant: return launch_mode<kRequant, FEAT>(f, volt, scale, out, power, st);
        case kPower: return launch_mode<kPower, FEAT>(f, volt, scale, out, power, st);
        case kRequantPlanar: return launch_mode<kRequantPlanar, FEAT>(f, volt, scale, out, power, st);
        default: return CORR_EINVAL;
    }
}

}  // namespace

// Per-feature entry points, one translation unit each.
corr_status fengine_run_plain(int mode, const FShape &f, const void *volt, const float *scale, void *out,
                              double *power, cudaStream_t st);
corr_status fengine_run_delay(int mode, const FShape &f, const void *volt, const float *scale, void *out,
                              double *power, cudaStream_t st);

}  // namespace corr
