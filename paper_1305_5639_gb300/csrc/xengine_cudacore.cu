// X-engine on CUDA cores (Eq. 2, Section 2): the plain baseline and the FP32 path.
//
// One CTA computes a 64 x 64 block of input pairs (I-block >= J-block, the lower
// triangle of Section 4) for one channel; 256 threads each own a 4 x 4 register
// block of pairs. Spectra are staged in shared memory in chunks, transposed to
// [spectrum][input] so that every thread reads broadcast / conflict-free.
//
//   FP32:  float2 input, V_ij += x_i conj(x_j) with FP32 FFMA.
//   INT8:  complex int8 input, exact INT32 result with dp4a: a 32-bit word holds
//          (re, im) of two consecutive spectra, so
//            Re V_ij += dp4a([re_i im_i ...], [re_j im_j ...])
//            Im V_ij += dp4a([im_i ~re_i ...], [re_j im_j ...]) + sum(im_j)
//          with ~re = -re - 1 (bitwise not), representable for every int8 code
//          including -128 (whose negation is not): the -1 terms sum to -sum(im_j),
//          which a per-column dp4a with [0 1 0 1] adds back.
#include "internal.h"

namespace corr {
namespace {

constexpr int TB = 64;          // inputs per tile side
constexpr int NTH = 256;        // threads (16 x 16)
constexpr int KC_F = 16;        // spectra per chunk, FP32
constexpr int KC_I = 32;        // spectra per chunk, INT8 (16 words)
constexpr int PAD = TB + 1;

__device__ __forceinline__ void tile_of(int t, int &bi, int &bj) {
    // t -> (bi, bj), bi >= bj, row-major over the lower triangle of blocks
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    bi = r;
    bj = t - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(NTH) k_xeng_f32(const float2 *__restrict__ X, float2 *__restrict__ acc,
                                                  const float2 *__restrict__ gains, int n_in, int K,
                                                  long long B, int store) {
    __shared__ float2 si[KC_F][PAD];
    __shared__ float2 sj[KC_F][PAD];
    int bi, bj;
    tile_of(blockIdx.x, bi, bj);
    const int chan = blockIdx.y;
    const int I0 = bi * TB, J0 = bj * TB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const float2 *Xc = X + (size_t)chan * n_in * K;

    float ar[4][4], ai[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) ar[r][c] = ai[r][c] = 0.0f;

    for (int a0 = 0; a0 < K; a0 += KC_F) {
#pragma unroll
        for (int q = 0; q < (TB * KC_F) / NTH; ++q) {
            int e = threadIdx.x + NTH * q;
            int row = e / KC_F, a = e % KC_F;
            int gi = I0 + row, gj = J0 + row, ga = a0 + a;
            float2 z = make_float2(0.f, 0.f);
            si[a][row] = (gi < n_in && ga < K) ? __ldg(Xc + (size_t)gi * K + ga) : z;
            sj[a][row] = (gj < n_in && ga < K) ? __ldg(Xc + (size_t)gj * K + ga) : z;
        }
        __syncthreads();
#pragma unroll 4
        for (int a = 0; a < KC_F; ++a) {
            float2 xi[4], xj[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) xi[r] = si[a][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) xj[c] = sj[a][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // x_i conj(x_j)
                    ar[r][c] = fmaf(xi[r].x, xj[c].x, fmaf(xi[r].y, xj[c].y, ar[r][c]));
                    ai[r][c] = fmaf(xi[r].y, xj[c].x, fmaf(-xi[r].x, xj[c].y, ai[r][c]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int i = I0 + ty + 16 * r;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int j = J0 + tx + 16 * c;
            if (i < n_in && j <= i) {
                float2 v = make_float2(ar[r][c], ai[r][c]);
                if (gains) {
                    float2 gi = __ldg(gains + i), gj = __ldg(gains + j);
                    // g_i conj(g_j)
                    float2 w = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
                    v = make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
                }
                size_t b = (size_t)chan * B + (size_t)i * (i + 1) / 2 + j;
                if (store) {
                    acc[b] = v;
                } else {
                    float2 o = acc[b];
                    acc[b] = make_float2(o.x + v.x, o.y + v.y);
                }
            }
        }
    }
}

// Few inputs (n_in <= kSmallIn, at most 253 packed pairs): a 64 x 64 tile would leave
// most of its threads idle, so one CTA takes one channel and each thread one packed
// pair (i >= j), the channel's spectra staged in shared memory in chunks of kSmallKC
// as [spectrum][input]. Four partial sums per pair (spectra a = r mod 4) keep four
// independent FMA chains in flight; they are added in a fixed order at the end, so
// the result is run-to-run identical.
constexpr int kSmallIn = 22;
constexpr int kSmallKC = 64;

__global__ void __launch_bounds__(NTH) k_xeng_f32_small(const float2 *__restrict__ X, float2 *__restrict__ acc,
                                                        const float2 *__restrict__ gains, int n_in, int K,
                                                        long long B, int store) {
    __shared__ float2 sx[kSmallKC][kSmallIn + 1];
    const int chan = blockIdx.x;
    const int p = threadIdx.x;
    int i = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= p) ++i;
    while (i * (i + 1) / 2 > p) --i;
    const int j = p - i * (i + 1) / 2;
    const bool live = p < B;
    const float2 *Xc = X + (size_t)chan * n_in * K;
    float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    for (int a0 = 0; a0 < K; a0 += kSmallKC) {
        for (int e = threadIdx.x; e < n_in * kSmallKC; e += NTH) {
            const int r = e / kSmallKC, a = e % kSmallKC;
            sx[a][r] = a0 + a < K ? __ldg(Xc + (size_t)r * K + a0 + a) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (live) {
#pragma unroll 4
            for (int a = 0; a < kSmallKC; a += 4) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    // x_i conj(x_j)
                    const float2 xi = sx[a + r][i], xj = sx[a + r][j];
                    re[r] = fmaf(xi.x, xj.x, fmaf(xi.y, xj.y, re[r]));
                    im[r] = fmaf(xi.y, xj.x, fmaf(-xi.x, xj.y, im[r]));
                }
            }
        }
        __syncthreads();
    }
    if (!live) return;
    float2 v = make_float2((re[0] + re[1]) + (re[2] + re[3]), (im[0] + im[1]) + (im[2] + im[3]));
    if (gains) {
        const float2 gi = __ldg(gains + i), gj = __ldg(gains + j);
        // g_i conj(g_j)
        const float2 w = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
        v = make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
    }
    const size_t b = (size_t)chan * B + p;
    if (store) {
        acc[b] = v;
    } else {
        const float2 o = acc[b];
        acc[b] = make_float2(o.x + v.x, o.y + v.y);
    }
}

__device__ __forceinline__ uint32_t rot_word(uint32_t w) {
    // bytes [re0 im0 re1 im1] -> [im0 ~re0 im1 ~re1] (~re = -re - 1)
    const uint32_t sw = __byte_perm(w, 0u, 0x2301);  // [im0 re0 im1 re1]
    return sw ^ 0xff00ff00u;
}
// dp4a weights picking the imaginary bytes of a word: [0 1 0 1]
constexpr int kImOnes = 0x01000100;

__global__ void __launch_bounds__(NTH) k_xeng_i8(const char2 *__restrict__ X, int2 *__restrict__ acc,
                                                 int n_in, int K, long long B, int store) {
    constexpr int KW = KC_I / 2;  // words per row per chunk
    __shared__ uint32_t si[KW][PAD];
    __shared__ uint32_t sr[KW][PAD];
    __shared__ uint32_t sj[KW][PAD];
    int bi, bj;
    tile_of(blockIdx.x, bi, bj);
    const int chan = blockIdx.y;
    const int I0 = bi * TB, J0 = bj * TB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const char2 *Xc = X + (size_t)chan * n_in * K;

    int ar[4][4], ai[4][4];
    int cim[4] = {0, 0, 0, 0};  // sum of Im x_j over the spectra, per column
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) ar[r][c] = ai[r][c] = 0;

    for (int a0 = 0; a0 < K; a0 += KC_I) {
#pragma unroll
        for (int q = 0; q < (TB * KW) / NTH; ++q) {
            int e = threadIdx.x + NTH * q;
            int row = e / KW, w = e % KW;
            int gi = I0 + row, gj = J0 + row, ga = a0 + 2 * w;
            uint32_t vi = 0, vj = 0;
            if (gi < n_in) {
                const char2 *p = Xc + (size_t)gi * K + ga;
                char2 c0 = ga < K ? p[0] : make_char2(0, 0);
                char2 c1 = ga + 1 < K ? p[1] : make_char2(0, 0);
                vi = (uint32_t)(uint8_t)c0.x | ((uint32_t)(uint8_t)c0.y << 8) | ((uint32_t)(uint8_t)c1.x << 16) |
                     ((uint32_t)(uint8_t)c1.y << 24);
            }
            if (gj < n_in) {
                const char2 *p = Xc + (size_t)gj * K + ga;
                char2 c0 = ga < K ? p[0] : make_char2(0, 0);
                char2 c1 = ga + 1 < K ? p[1] : make_char2(0, 0);
                vj = (uint32_t)(uint8_t)c0.x | ((uint32_t)(uint8_t)c0.y << 8) | ((uint32_t)(uint8_t)c1.x << 16) |
                     ((uint32_t)(uint8_t)c1.y << 24);
            }
            si[w][row] = vi;
            sr[w][row] = rot_word(vi);
            sj[w][row] = vj;
        }
        __syncthreads();
#pragma unroll 4
        for (int w = 0; w < KW; ++w) {
            int xi[4], xr[4], xj[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                xi[r] = (int)si[w][ty + 16 * r];
                xr[r] = (int)sr[w][ty + 16 * r];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                xj[c] = (int)sj[w][tx + 16 * c];
                cim[c] = __dp4a(xj[c], kImOnes, cim[c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    ar[r][c] = __dp4a(xi[r], xj[c], ar[r][c]);
                    ai[r][c] = __dp4a(xr[r], xj[c], ai[r][c]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int i = I0 + ty + 16 * r;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int j = J0 + tx + 16 * c;
            if (i < n_in && j <= i) {
                size_t b = (size_t)chan * B + (size_t)i * (i + 1) / 2 + j;
                const int im = ai[r][c] + cim[c];
                if (store) {
                    acc[b] = make_int2(ar[r][c], im);
                } else {
                    int2 o = acc[b];
                    acc[b] = make_int2(o.x + ar[r][c], o.y + im);
                }
            }
        }
    }
}

}  // namespace

corr_status launch_xengine_cudacore(const Handle &h, const void *chan_in, const float2 *gains, bool store,
                                    cudaStream_t st) {
    const int nb = (h.n_in + TB - 1) / TB;
    dim3 grid(nb * (nb + 1) / 2, h.n_chan);
    StageScope sc(h, CORR_STAGE_XENGINE, st);
    if (h.precision == CORR_PREC_INT8) {
        k_xeng_i8<<<grid, NTH, 0, st>>>(static_cast<const char2 *>(chan_in), static_cast<int2 *>(h.acc), h.n_in,
                                        h.n_spectra, h.n_base, store ? 1 : 0);
    } else if (h.n_in <= kSmallIn) {
        k_xeng_f32_small<<<h.n_chan, NTH, 0, st>>>(static_cast<const float2 *>(chan_in),
                                                   static_cast<float2 *>(h.acc), gains, h.n_in, h.n_spectra,
                                                   h.n_base, store ? 1 : 0);
    } else {
        k_xeng_f32<<<grid, NTH, 0, st>>>(static_cast<const float2 *>(chan_in), static_cast<float2 *>(h.acc),
                                         gains, h.n_in, h.n_spectra, h.n_base, store ? 1 : 0);
    }
    return check_launch("k_xeng_cudacore");
}

}  // namespace corr
