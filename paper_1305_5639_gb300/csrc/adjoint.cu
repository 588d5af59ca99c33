// Adjoint of the gained X-engine for gradient-based gain calibration.
//
// Forward (per channel f): V'_ij = g_i conj(g_j) sum_a X_ia conj(X_ja), i >= j.
// Given G = dL/dV' (PyTorch convention, packed i >= j) and its Hermitian
// completion G^ (G^_ij = G_ij for i > j, G^_ji = conj G_ij, G^_ii = 2 Re G_ii):
//     Y      = G^ diag(g) X                      (complex GEMM, n_in x n_in x K)
//     dL/dX  = diag(conj g) Y
//     dL/dg_m = sum_f sum_a conj(X_ma) Y_ma      (= sum_f sum_j G^_mj g_j V_jm)
// The dg reduction is fused into the GEMM epilogue: each CTA writes one partial
// per row into a workspace, and a second kernel sums the partials in a fixed
// order (bit-reproducible).
#include "internal.h"

namespace corr {
namespace {

constexpr int TM = 64, TA = 64, JC = 16, NTH = 256;

__device__ __forceinline__ float2 ghat(const float2 *__restrict__ G, int m, int j, int n_in) {
    if (m >= n_in || j >= n_in) return make_float2(0.f, 0.f);
    if (m > j) return __ldg(G + (size_t)m * (m + 1) / 2 + j);
    if (m < j) {
        float2 v = __ldg(G + (size_t)j * (j + 1) / 2 + m);
        return make_float2(v.x, -v.y);
    }
    float2 v = __ldg(G + (size_t)m * (m + 1) / 2 + m);
    return make_float2(2.0f * v.x, 0.0f);
}

__global__ void __launch_bounds__(NTH) k_adj(const float2 *__restrict__ Gp, const float2 *__restrict__ X,
                                             const float2 *__restrict__ gains, float2 *__restrict__ dX,
                                             float2 *__restrict__ part, int n_in, int K, long long B) {
    __shared__ float2 sg[JC][TM + 1];  // sg[jj][m] = G^_{m, j}
    __shared__ float2 sz[JC][TA + 1];  // sz[jj][a] = g_j X_{j, a}
    const int M0 = blockIdx.x * TM, A0 = blockIdx.y * TA, chan = blockIdx.z;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const float2 *Gc = Gp + (size_t)chan * B;
    const float2 *Xc = X + (size_t)chan * n_in * K;

    float yr[4][4], yi[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) yr[r][c] = yi[r][c] = 0.f;

    for (int j0 = 0; j0 < n_in; j0 += JC) {
#pragma unroll
        for (int q = 0; q < (TM * JC) / NTH; ++q) {
            int e = threadIdx.x + NTH * q;
            int ml = e / JC, jj = e % JC;
            sg[jj][ml] = ghat(Gc, M0 + ml, j0 + jj, n_in);
        }
#pragma unroll
        for (int q = 0; q < (TA * JC) / NTH; ++q) {
            int e = threadIdx.x + NTH * q;
            int jj = e / TA, al = e % TA;
            int j = j0 + jj, a = A0 + al;
            float2 z = make_float2(0.f, 0.f);
            if (j < n_in && a < K) {
                float2 x = __ldg(Xc + (size_t)j * K + a);
                float2 g = gains ? __ldg(gains + j) : make_float2(1.f, 0.f);
                z = make_float2(g.x * x.x - g.y * x.y, g.x * x.y + g.y * x.x);
            }
            sz[jj][al] = z;
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < JC; ++jj) {
            float2 gv[4], zv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) gv[r] = sg[jj][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) zv[c] = sz[jj][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    yr[r][c] = fmaf(gv[r].x, zv[c].x, fmaf(-gv[r].y, zv[c].y, yr[r][c]));
                    yi[r][c] = fmaf(gv[r].x, zv[c].y, fmaf(gv[r].y, zv[c].x, yi[r][c]));
                }
        }
        __syncthreads();
    }

    // epilogue: dX = conj(g_m) Y, partial dg_m = sum_a conj(X_ma) Y_ma
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int m = M0 + ty + 16 * r;
        float pr = 0.f, pi = 0.f;
        if (m < n_in) {
            float2 g = gains ? __ldg(gains + m) : make_float2(1.f, 0.f);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int a = A0 + tx + 16 * c;
                if (a < K) {
                    float2 x = __ldg(Xc + (size_t)m * K + a);
                    float2 y = make_float2(yr[r][c], yi[r][c]);
                    // conj(x) y
                    pr = fmaf(x.x, y.x, fmaf(x.y, y.y, pr));
                    pi = fmaf(x.x, y.y, fmaf(-x.y, y.x, pi));
                    if (dX) {
                        // conj(g) y
                        dX[((size_t)chan * n_in + m) * K + a] =
                            make_float2(g.x * y.x + g.y * y.y, g.x * y.y - g.y * y.x);
                    }
                }
            }
        }
        if (part) {
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {
                pr += __shfl_xor_sync(0xffffffffu, pr, off);
                pi += __shfl_xor_sync(0xffffffffu, pi, off);
            }
            if (tx == 0 && m < n_in)
                part[((size_t)chan * gridDim.y + blockIdx.y) * n_in + m] = make_float2(pr, pi);
        }
    }
}

// dL/dg = sum of n_part per-row partials, in two fixed-order levels (bit-reproducible):
// level 1 sums the partials of kRedSplit contiguous ranges in FP64, level 2 the ranges.
constexpr int kRedSplit = 64;

__global__ void k_adj_reduce1(const float2 *__restrict__ part, double2 *__restrict__ mid, int n_in, long long n_part) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_in) return;
    const long long per = (n_part + kRedSplit - 1) / kRedSplit;
    const long long p0 = per * blockIdx.y, p1 = min(n_part, p0 + per);
    double sr = 0.0, si = 0.0;
    for (long long q = p0; q < p1; ++q) {
        const float2 v = __ldg(part + q * n_in + m);
        sr += v.x;
        si += v.y;
    }
    mid[(size_t)blockIdx.y * n_in + m] = make_double2(sr, si);
}

__global__ void k_adj_reduce2(const double2 *__restrict__ mid, float2 *__restrict__ dg, int n_in) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_in) return;
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < kRedSplit; ++s) {
        const double2 v = mid[(size_t)s * n_in + m];
        sr += v.x;
        si += v.y;
    }
    dg[m] = make_float2((float)sr, (float)si);
}

}  // namespace

size_t backward_workspace_bytes(const Handle &h) {
    const int nA = (h.n_spectra + TA - 1) / TA;
    return align16(sizeof(float2) * (size_t)h.n_chan * nA * h.n_in) + adj_reduce_scratch_bytes(h.n_in);
}

size_t adj_reduce_scratch_bytes(int n_in) { return sizeof(double2) * (size_t)kRedSplit * n_in; }

corr_status launch_backward_ws(const Handle &h, const float2 *grad_vis, const float2 *chan_in,
                               const float2 *gains, float2 *grad_chan, float2 *grad_gains, float2 *ws,
                               cudaStream_t st) {
    const int nM = (h.n_in + TM - 1) / TM, nA = (h.n_spectra + TA - 1) / TA;
    if (h.n_chan > 65535) return CORR_EUNSUPPORTED;
    dim3 grid(nM, nA, h.n_chan);
    corr_status s;
    {
        StageScope sc(h, CORR_STAGE_ADJ_GEMM, st);
        k_adj<<<grid, NTH, 0, st>>>(grad_vis, chan_in, gains, grad_chan, grad_gains ? ws : nullptr, h.n_in,
                                    h.n_spectra, h.n_base);
        s = check_launch("k_adj");
    }
    if (s != CORR_OK || !grad_gains) return s;
    const long long n_part = (long long)h.n_chan * nA;
    double2 *scratch = reinterpret_cast<double2 *>(reinterpret_cast<char *>(ws) +
                                                   align16(sizeof(float2) * (size_t)n_part * h.n_in));
    StageScope sc(h, CORR_STAGE_ADJ_REDUCE, st, 2);
    return launch_adj_reduce(ws, scratch, grad_gains, h.n_in, n_part, st);
}

corr_status launch_adj_reduce(const float2 *part, double2 *scratch, float2 *dg, int n_in, long long n_part,
                              cudaStream_t st) {
    const unsigned nb = (unsigned)((n_in + 127) / 128);
    k_adj_reduce1<<<dim3(nb, kRedSplit), 128, 0, st>>>(part, scratch, n_in, n_part);
    corr_status s = check_launch("k_adj_reduce1");
    if (s != CORR_OK) return s;
    k_adj_reduce2<<<nb, 128, 0, st>>>(scratch, dg, n_in);
    return check_launch("k_adj_reduce2");
}

}  // namespace corr
