// Integration dump: the long-integration FP64 buffer receives the integration
// accumulator (INT32 pairs for INT8, FP32 pairs otherwise) in one streaming pass
// (read 8 B + read/write 16 B per visibility), with the FP64 pipe doing at most the
// add itself (exact_add.cuh: INT32 sums are added in integers, FP32 sums converted
// in integers). The accumulator is not
// rewritten with zeros: the handle marks it clear, so the next X-engine launch
// overwrites it instead of adding to it and corr_get_accum returns zeros meanwhile.
#include "exact_add.cuh"
#include "internal.h"

namespace corr {
namespace {

template <typename AccT>
__global__ void __launch_bounds__(256) k_dump(const AccT *__restrict__ acc, double2 *__restrict__ vis, long long n) {
    // four visibilities per thread and round, all loads before any store (more bytes in
    // flight per thread for the read-modify-write of the FP64 buffer)
    constexpr int U = 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e + (U - 1) * stride < n; e += U * stride) {
        AccT a[U];
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] = __ldcs(acc + e + u * stride);
            v[u] = vis[e + u * stride];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) vis[e + u * stride] = add_exact(v[u], a[u]);
    }
    for (; e < n; e += stride) vis[e] = add_exact(vis[e], __ldcs(acc + e));
}

}  // namespace

corr_status launch_dump(const Handle &h, cudaStream_t st) { return launch_dump_range(h, 0, h.n_chan, st); }

corr_status launch_dump_src(const Handle &h, const void *acc, cudaStream_t st) {
    const long long n = (long long)h.n_chan * h.n_base;
    if (n <= 0) return CORR_OK;
    StageScope sc(h, CORR_STAGE_DUMP, st);
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)h.n_sm * 16;
    if (blocks > cap) blocks = cap;
    if (h.precision == CORR_PREC_INT8)
        k_dump<int2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const int2 *>(acc), h.vis64, n);
    else
        k_dump<float2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const float2 *>(acc), h.vis64, n);
    return check_launch("k_dump");
}

corr_status launch_dump_range(const Handle &h, int c0, int c1, cudaStream_t st) {
    const long long n = (long long)(c1 - c0) * h.n_base;
    if (n <= 0) return CORR_OK;
    const long long off = (long long)c0 * h.n_base;
    StageScope sc(h, CORR_STAGE_DUMP, st);
    long long blocks = (n + 255) / 256;
    const long long cap = (long long)h.n_sm * 16;
    if (blocks > cap) blocks = cap;
    if (h.precision == CORR_PREC_INT8)
        k_dump<int2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<int2 *>(h.acc) + off, h.vis64 + off, n);
    else
        k_dump<float2><<<(unsigned)blocks, 256, 0, st>>>(static_cast<float2 *>(h.acc) + off, h.vis64 + off, n);
    return check_launch("k_dump");
}

}  // namespace corr
