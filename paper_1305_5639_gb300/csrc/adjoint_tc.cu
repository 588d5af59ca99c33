// Adjoint of the gained X-engine on tcgen05 tensor cores, FP16 hi/lo split
// (gradient-based gain calibration through Eq. 2 of Section 2).
//
// Per channel f, with G^_f the Hermitian completion of the packed gradient G_f
// (G^_ij = G_ij for i > j, G^_ji = conj G_ij, G^_ii = 2 Re G_ii):
//     A_f   = 2^e_f G^_f diag(g)                        n_in x n_in
//     Y_f   = 2^-e_f A_f X_f                            (dX GEMM, tensor cores)
//     dL/dX_f = diag(conj g) Y_f,   dL/dg_m = sum_f sum_a conj(X_f,ma) Y_f,ma
// The power-of-two scale e_f brings A_f into FP16's normal range (the packed
// gradient of a loss over visibilities normalised by the integration length is
// typically ~1e-6); it is exact and undone in the GEMM epilogue. Both operands are
// split x = h + l with h = fp16(x), l = fp16(x - h) and the products taken as
// hh + hl + lh (the X-engine's hi/lo scheme). X_f itself is not rescaled, so the
// channelised data are expected within FP16's normal range, as for the forward
// FP16 paths.
//
// Passes:
//   k_adj_expo   e_f from max |G_f| and max |g|, all channels   reads G once
// then per block of channels, the operand passes of the next block on a side stream
// overlapping the GEMM of the current one (two operand buffers):
//   k_adj_aprep  A_f planes [f][Re_h, Im_h, Re_l, Im_l][m][j]   reads G, writes 8 B / entry
//   k_adj_bprep  X_f^T planes [f][4][a][j]                  reads X, writes 8 B / sample
//   k_xeng_tma<kAdj>  GEMM + epilogue (dX, dg partials)
// and one fixed-order reduction of the dg partials over all channels.
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.h"

namespace corr {
namespace {

__device__ __forceinline__ void split_hl(float x, __half &h, __half &l) {
    h = __float2half_rn(x);
    l = __float2half_rn(x - __half2float(h));
}

// e_f = 15 - k with bound(f) < 2^k, bound = 3 max|G_f| max|g| (>= every |Re|, |Im| of A_f / 2^e_f)
__global__ void __launch_bounds__(256) k_adj_expo(const float2 *__restrict__ Gp, const float2 *__restrict__ gains,
                                                  int *__restrict__ expo, int n_in, long long B, int c0) {
    __shared__ float red[2][8];
    const float2 *G = Gp + (size_t)(c0 + blockIdx.x) * B;
    float mg = 0.f, mq = gains ? 0.f : 1.f;
    for (long long b = threadIdx.x; b < B; b += blockDim.x) {
        const float2 v = __ldg(G + b);
        mg = fmaxf(mg, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    if (gains)
        for (int j = threadIdx.x; j < n_in; j += blockDim.x) {
            const float2 v = __ldg(gains + j);
            mq = fmaxf(mq, sqrtf(v.x * v.x + v.y * v.y));
        }
    for (int o = 16; o > 0; o >>= 1) {
        mg = fmaxf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
        mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = mg;
        red[1][threadIdx.x >> 5] = mq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mg = fmaxf(mg, red[0][w]);
            mq = fmaxf(mq, red[1][w]);
        }
        const float bound = 3.0f * mg * mq;
        int e = 0;
        if (bound > 0.f && isfinite(bound)) {
            int k = 0;
            frexpf(bound, &k);  // bound < 2^k
            e = min(100, max(-100, 15 - k));
        }
        expo[blockIdx.x] = e;
    }
}

// The operand passes move 64 x 64 tiles through shared memory (rows padded to 65
// complex values) and write each output row as 16-byte pieces of 8 consecutive
// columns per plane, 8 threads per row.
constexpr int kPT = 64;   // prep tile edge
constexpr int kPTS = 65;  // padded row stride of the shared tile (complex values)

// 8 complex values -> the 4 FP16 planes (Re_h, Im_h, Re_l, Im_l), 16 bytes each.
__device__ __forceinline__ void store8_planes(const float (&re)[8], const float (&im)[8], __half *dst,
                                              size_t plane) {
    uint32_t w[4][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        __half rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
        split_hl(re[q], rh0, rl0);
        split_hl(im[q], ih0, il0);
        split_hl(re[q + 1], rh1, rl1);
        split_hl(im[q + 1], ih1, il1);
        w[0][q / 2] = (uint32_t)__half_as_ushort(rh0) | ((uint32_t)__half_as_ushort(rh1) << 16);
        w[1][q / 2] = (uint32_t)__half_as_ushort(ih0) | ((uint32_t)__half_as_ushort(ih1) << 16);
        w[2][q / 2] = (uint32_t)__half_as_ushort(rl0) | ((uint32_t)__half_as_ushort(rl1) << 16);
        w[3][q / 2] = (uint32_t)__half_as_ushort(il0) | ((uint32_t)__half_as_ushort(il1) << 16);
    }
#pragma unroll
    for (int pl = 0; pl < 4; ++pl)
        *reinterpret_cast<uint4 *>(dst + pl * plane) = make_uint4(w[pl][0], w[pl][1], w[pl][2], w[pl][3]);
}

// A_f = 2^e_f G^_f diag(g) as four FP16 planes [f - c0][plane][m][j]. One CTA per
// lower-triangle tile (mb >= jb) of 64 x 64 entries: the packed gradient's tile
// T[r][c] = G(m0 + r, j0 + c) is read once and gives both A tiles it defines:
//   tile (mb, jb):  A[m][j] = G^_mj g_j with G^_mj = T[r][c] (on the diagonal tile:
//                   conj T[c][r] above the diagonal, 2 Re T[r][r] on it)
//   tile (jb, mb):  A[j][m] = conj(T[r][c]) g_m      (mb > jb only)
// n_in must be a multiple of 8 (whole 16-byte pieces).
__global__ void __launch_bounds__(256) k_adj_aprep(const float2 *__restrict__ Gp, const float2 *__restrict__ gains,
                                                   const int *__restrict__ expo, __half *__restrict__ A, int n_in,
                                                   long long B, int c0) {
    __shared__ float2 T[kPT * kPTS];
    const int t = blockIdx.x, fl = blockIdx.y;
    int mb = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((mb + 1) * (mb + 2) / 2 <= t) ++mb;
    while (mb * (mb + 1) / 2 > t) --mb;
    const int jb = t - mb * (mb + 1) / 2;
    const float2 *G = Gp + (size_t)(c0 + fl) * B;
    const int m0 = mb * kPT, j0 = jb * kPT;
    const bool diag = mb == jb;
    for (int e = threadIdx.x; e < kPT * kPT; e += blockDim.x) {
        const int r = e / kPT, c = e % kPT;
        const int m = m0 + r, j = j0 + c;
        float2 v = make_float2(0.f, 0.f);
        if (m < n_in && j < n_in && (!diag || c <= r)) v = __ldg(G + (size_t)m * (m + 1) / 2 + j);
        T[r * kPTS + c] = v;
    }
    __syncthreads();
    const float sc = ldexpf(1.0f, __ldg(expo + fl));
    const size_t plane = (size_t)n_in * n_in;
    __half *Af = A + (size_t)fl * 4 * plane;
    // 64 rows x 8 pieces of 8 columns per output tile, two (row, piece) items per thread
    for (int it = threadIdx.x; it < kPT * 8; it += blockDim.x) {
        const int r = it / 8, ch = it % 8;
        // tile (mb, jb): row m = m0 + r, columns j = j0 + 8 ch + q
        const int m = m0 + r, jc = j0 + 8 * ch;
        if (m < n_in && jc < n_in) {
            float re[8], im[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = 8 * ch + q;
                float2 gh;
                if (!diag || r > c) gh = T[r * kPTS + c];
                else if (r < c) gh = make_float2(T[c * kPTS + r].x, -T[c * kPTS + r].y);
                else gh = make_float2(2.0f * T[r * kPTS + r].x, 0.0f);
                const float2 g = gains ? __ldg(gains + jc + q) : make_float2(1.f, 0.f);
                re[q] = (gh.x * g.x - gh.y * g.y) * sc;
                im[q] = (gh.x * g.y + gh.y * g.x) * sc;
            }
            store8_planes(re, im, Af + (size_t)m * n_in + jc, plane);
        }
        // tile (jb, mb): row j = j0 + r, columns m = m0 + 8 ch + q, A[j][m] = conj(G(m, j)) g_m
        const int j = j0 + r, mc = m0 + 8 * ch;
        if (!diag && j < n_in && mc < n_in) {
            float re[8], im[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float2 v = T[(8 * ch + q) * kPTS + r];  // G(m, j), m = mc + q
                const float2 g = gains ? __ldg(gains + mc + q) : make_float2(1.f, 0.f);
                re[q] = (v.x * g.x + v.y * g.y) * sc;  // conj(v) g
                im[q] = (v.x * g.y - v.y * g.x) * sc;
            }
            store8_planes(re, im, Af + (size_t)j * n_in + mc, plane);
        }
    }
}

// X_f^T as four FP16 planes [f - c0][plane][a][j]: one CTA per 64 inputs j x 64
// spectra a, read as 16-byte pairs of spectra, transposed through shared memory.
// n_in and K must be multiples of 8.
__global__ void __launch_bounds__(256) k_adj_bprep(const float2 *__restrict__ X, __half *__restrict__ Bt, int n_in,
                                                   int K, int c0) {
    __shared__ float2 T[kPT * kPTS];  // T[j][a]
    const int ab = blockIdx.x, jb = blockIdx.y, fl = blockIdx.z;
    const int j0 = jb * kPT, a0 = ab * kPT;
    const float2 *Xc = X + (size_t)(c0 + fl) * n_in * K;
    for (int e = threadIdx.x; e < kPT * kPT / 2; e += blockDim.x) {
        const int r = e / (kPT / 2), c = 2 * (e % (kPT / 2));
        const int j = j0 + r, a = a0 + c;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n_in && a < K) v = __ldg(reinterpret_cast<const float4 *>(Xc + (size_t)j * K + a));
        T[r * kPTS + c] = make_float2(v.x, v.y);
        T[r * kPTS + c + 1] = make_float2(v.z, v.w);
    }
    __syncthreads();
    const size_t plane = (size_t)K * n_in;
    __half *Bf = Bt + (size_t)fl * 4 * plane;
    for (int it = threadIdx.x; it < kPT * 8; it += blockDim.x) {
        const int r = it / 8, ch = it % 8;  // output row a = a0 + r, columns j = j0 + 8 ch + q
        const int a = a0 + r, jc = j0 + 8 * ch;
        if (a >= K || jc >= n_in) continue;
        float re[8], im[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float2 x = T[(8 * ch + q) * kPTS + r];
            re[q] = x.x;
            im[q] = x.y;
        }
        store8_planes(re, im, Bf + (size_t)a * n_in + jc, plane);
    }
}

// Workspace layout: [dg partials][reduce scratch][exponents][A planes][B planes],
// the planes sized for one block of chan_block channels.
struct TcWs {
    size_t part, scratch, expo, a[2], b[2], total;
    int cb;
};

constexpr size_t kPlaneBudget = (size_t)1 << 30;  // operand planes of one channel block

TcWs tc_layout(const Handle &h) {
    TcWs w{};
    const int nbj = (h.n_spectra + 127) / 128;
    const size_t per_chan = 8ull * h.n_in * h.n_in + 8ull * h.n_spectra * h.n_in;  // A + B planes
    const int cb_max = (int)std::max<size_t>(1, std::min<size_t>((size_t)h.n_chan, kPlaneBudget / per_chan));
    const int n_blk = (h.n_chan + cb_max - 1) / cb_max;
    w.cb = (h.n_chan + n_blk - 1) / n_blk;  // balanced blocks
    size_t o = 0;
    w.part = o;
    o += align16(sizeof(float2) * (size_t)h.n_chan * nbj * 2 * h.n_in);
    w.scratch = o;
    o += align16(adj_reduce_scratch_bytes(h.n_in));
    w.expo = o;
    o += sizeof(int) * (size_t)h.n_chan;
    for (int k = 0; k < 2; ++k) {  // two buffers: block b + 1 is prepared while block b's GEMM runs
        o = (o + 1023) & ~(size_t)1023;
        w.a[k] = o;
        o += align16(8ull * w.cb * h.n_in * h.n_in);
        o = (o + 1023) & ~(size_t)1023;
        w.b[k] = o;
        o += align16(8ull * w.cb * h.n_spectra * h.n_in);
    }
    w.total = o;
    return w;
}

}  // namespace

size_t backward_tc_workspace_bytes(const Handle &h, int *chan_block) {
    const TcWs w = tc_layout(h);
    if (chan_block) *chan_block = w.cb;
    return w.total;
}

// The operand passes of block b + 1 run on the side stream `side` while block b's GEMM
// runs on `st`; ev[0] orders the side stream after `st`'s earlier work, ev[1 + k]
// marks buffer k prepared, ev[3 + k] buffer k consumed.
corr_status launch_backward_tc(const Handle &h, const float2 *grad_vis, const float2 *chan_in, const float2 *gains,
                               float2 *grad_chan, float2 *grad_gains, void *ws, cudaStream_t st,
                               cudaStream_t side, cudaEvent_t *ev) {
    if ((h.n_in % 8) != 0 || (h.n_spectra % 8) != 0) return CORR_EUNSUPPORTED;
    if (h.n_chan > 65535) return CORR_EUNSUPPORTED;
    const TcWs w = tc_layout(h);
    char *base = static_cast<char *>(ws);
    float2 *part = grad_gains ? reinterpret_cast<float2 *>(base + w.part) : nullptr;
    int *expo = reinterpret_cast<int *>(base + w.expo);
    const int nt_in = (h.n_in + kPT - 1) / kPT, nt_k = (h.n_spectra + kPT - 1) / kPT;
    const int n_tri = nt_in * (nt_in + 1) / 2;
    CORR_CUDA_TRY(cudaEventRecord(ev[0], st));
    CORR_CUDA_TRY(cudaStreamWaitEvent(side, ev[0], 0));
    corr_status s;
    {
        StageScope sc(h, CORR_STAGE_ADJ_PREP, side);
        k_adj_expo<<<h.n_chan, 256, 0, side>>>(grad_vis, gains, expo, h.n_in, h.n_base, 0);
        s = check_launch("k_adj_expo");
    }
    if (s != CORR_OK) return s;
    int blk = 0;
    for (int c0 = 0; c0 < h.n_chan; c0 += w.cb, ++blk) {
        const int c1 = std::min(h.n_chan, c0 + w.cb), nc = c1 - c0, k = blk & 1;
        __half *A = reinterpret_cast<__half *>(base + w.a[k]);
        __half *Bt = reinterpret_cast<__half *>(base + w.b[k]);
        if (blk >= 2) CORR_CUDA_TRY(cudaStreamWaitEvent(side, ev[3 + k], 0));  // GEMM of block - 2 done
        {
            StageScope sc(h, CORR_STAGE_ADJ_PREP, side, 2);
            k_adj_aprep<<<dim3(n_tri, nc), 256, 0, side>>>(grad_vis, gains, expo + c0, A, h.n_in, h.n_base, c0);
            if ((s = check_launch("k_adj_aprep")) != CORR_OK) return s;
            k_adj_bprep<<<dim3(nt_k, nt_in, nc), 256, 0, side>>>(chan_in, Bt, h.n_in, h.n_spectra, c0);
            if ((s = check_launch("k_adj_bprep")) != CORR_OK) return s;
        }
        CORR_CUDA_TRY(cudaEventRecord(ev[1 + k], side));
        CORR_CUDA_TRY(cudaStreamWaitEvent(st, ev[1 + k], 0));
        s = launch_adjoint_tma(h, A, Bt, expo + c0, chan_in, gains, grad_chan, part, c0, c1, st);
        if (s != CORR_OK) return s;
        CORR_CUDA_TRY(cudaEventRecord(ev[3 + k], st));
    }
    if (!grad_gains) return CORR_OK;
    const int nbj = (h.n_spectra + 127) / 128;
    StageScope sc(h, CORR_STAGE_ADJ_REDUCE, st, 2);
    return launch_adj_reduce(part, reinterpret_cast<double2 *>(base + w.scratch), grad_gains, h.n_in,
                             (long long)h.n_chan * nbj * 2, st);
}

}  // namespace corr
