// Integration dump: the long-integration FP64 buffer receives the integration
// accumulator (INT32 pairs for INT8, FP32 pairs otherwise) in one streaming pass
// (read 8 B + read/write 16 B per visibility). The accumulator is not
// rewritten with zeros: the handle marks it clear, so the next X-engine launch
// overwrites it instead of adding to it and corr_get_accum returns zeros meanwhile.
#include "internal.h"

namespace corr {
namespace {

// ---- exact integer arithmetic on integer-valued doubles (INT8 path)
// The INT8 long integration holds exact integers (sums of INT32 dumps), and GB300's
// FP64 path is slow, so the integer dump decodes each double to an int64, adds the
// INT32 partial and encodes the sum again, with integer instructions only. The
// result is bit-identical to the FP64 add: both are exact while |value| < 2^53, and
// any element outside that range, or not an integer, takes the FP64 add.

// v = m 2^(e - 1075) with the hidden bit in m; integer if the shifted-out bits are 0
__device__ __forceinline__ bool dbl_to_i64(unsigned long long b, long long &n) {
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) {  // +-0 (an integer sum has no subnormals)
        n = 0;
        return (b << 1) == 0;
    }
    const int sh = 1075 - e;
    if (sh < 1 || sh > 52) return false;  // |v| >= 2^52 or |v| < 1 (non-zero): FP64 path
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

__device__ __forceinline__ double2 add_int(double2 v, int2 a) {
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

__device__ __forceinline__ double2 add_acc(double2 v, int2 a) { return add_int(v, a); }
__device__ __forceinline__ double2 add_acc(double2 v, float2 a) {
    return make_double2(v.x + (double)a.x, v.y + (double)a.y);
}

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
        for (int u = 0; u < U; ++u) vis[e + u * stride] = add_acc(v[u], a[u]);
    }
    for (; e < n; e += stride) vis[e] = add_acc(vis[e], __ldcs(acc + e));
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
