// X-engine on the 5th-generation tensor cores (tcgen05, kind::f16), Eq. 2 of
// Section 2 as a Hermitian rank-K update V[f] += X[f] X[f]^H, lower triangle.
//
// Complex -> real mapping. For a tile of 128 inputs I (rows) x 128 inputs J, with
// per-spectrum planes re, im and a negated plane -im of the J block, two real MMAs
// of M = 128, N = 256, K = 16 per 16 spectra give
//     D[:, 0:128]   += re_I re_J^T + im_I im_J^T  = Re V_IJ
//     D[:, 128:256] += re_I (-im_J)^T + im_I re_J^T = Im V_IJ
// from A = re_I with B = [re_J ; -im_J] and A = im_I with B = [im_J ; re_J]. The J
// planes are stored [im | re | -im] so both B operands are contiguous 256-row
// slices. Diagonal tiles (I == J) reuse the J planes as A.
//
// INT8: int8 values (-128 included; its negation 128 too) are exact in FP16 and
// every product (<= 128^2) is exact in FP32; one accumulator column sums at most
// 2 * 128^2 * 512 = 2^24 in magnitude over 512 spectra, so FP32 partial sums of
// <= 512 spectra are exact integers. After each
// 512-spectrum chunk the epilogue adds the FP32 partial (converted exactly) into
// an INT32 running sum held in TMEM columns 256..511: the result is bit-exact.
// FP16: inputs rounded to FP16, FP32 accumulation over the whole integration, with
// the accumulator double-buffered in TMEM so the epilogue overlaps the next tile.
//
// Warp roles (544 threads, one persistent CTA per SM; 17 warps put 5 warps on one
// SM sub-partition, whose 16K-register file caps the kernel at 96 registers):
//   warps 0-7   producers: global loads (one stage ahead, in registers) -> FP16
//               planes in 128B-swizzled K-major shared memory
//   warp  8     TMEM allocator + single-thread MMA issuer
//   warps 9-16  epilogue, two warps per TMEM lane quarter (each half the columns):
//               tcgen05.ld -> (INT32 fold | gains) -> packed global store
// Every mbarrier wait is bounded; on time-out the CTA records CORR_ETIMEOUT and
// all roles leave their loops.
#include <cuda_fp16.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace corr {
namespace {

constexpr int TILE = 128;                  // inputs per tile side
constexpr int KB = 64;                     // spectra per pipeline stage (128 B of fp16 per row)
constexpr int BLK = TILE * KB * 2;         // one fp16 plane block: 16 KB
constexpr int NBLK = 5;                    // A_re, A_im, B_im, B_re, B_nim
constexpr int STAGE_BYTES = NBLK * BLK;    // 80 KB
constexpr int NSTAGE = 2;
constexpr int CHUNK_KB = 8;                // INT8 flush every 8 stages = 512 spectra
constexpr int NPW = 8;                     // producer warps
constexpr int MMA_WARP = NPW;              // TMEM allocator + MMA issuer
constexpr int NEW = 8;                     // epilogue warps (two per TMEM lane quarter)
constexpr int NPROD = 32 * NPW, NEPI = 32 * NEW;
constexpr int NTHREADS = NPROD + 32 + NEPI;
constexpr int OFF_ARE = 0, OFF_AIM = BLK, OFF_BIM = 2 * BLK, OFF_BRE = 3 * BLK, OFF_BNIM = 4 * BLK;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

enum XMode { kInt8 = 0, kFp16 = 1 };

struct XParams {
    const void *X;
    void *acc;
    const float2 *gains;
    int *status;
    long long B;
    long long n_items;
    int n_in, K, nb, n_tiles, store;
};

__device__ __forceinline__ void decode_item(long long item, int n_tiles, int &chan, int &bi, int &bj) {
    chan = (int)(item / n_tiles);
    int t = (int)(item % n_tiles);
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    bi = r;
    bj = t - r * (r + 1) / 2;
}

__device__ __forceinline__ uint32_t h2_sub(uint32_t a, uint32_t b) {
    __half2 x = *reinterpret_cast<__half2 *>(&a), y = *reinterpret_cast<__half2 *>(&b);
    __half2 z = __hsub2(x, y);
    return *reinterpret_cast<uint32_t *>(&z);
}

// 8 spectra of complex int8 (16 B) -> fp16 planes re, im, -im (16 B each).
__device__ __forceinline__ void cvt_i8(const uint4 &v, uint4 &re, uint4 &im, uint4 &nim) {
    const uint32_t K1152 = 0x64806480u;  // half2(1152, 1152)
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t r[4], i[4], n[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // x ^ 0x80 = x + 128 as unsigned; 0x64 in the high byte makes the half 1024 + u
        uint32_t u = w[q] ^ 0x80808080u;
        uint32_t hr = __byte_perm(u, 0x64646464u, 0x4240);
        uint32_t hi = __byte_perm(u, 0x64646464u, 0x4341);
        r[q] = h2_sub(hr, K1152);
        i[q] = h2_sub(hi, K1152);
        n[q] = h2_sub(K1152, hi);
    }
    re = make_uint4(r[0], r[1], r[2], r[3]);
    im = make_uint4(i[0], i[1], i[2], i[3]);
    nim = make_uint4(n[0], n[1], n[2], n[3]);
}

// 2 spectra of complex float (16 B) -> one fp16x2 of re, of im, of -im.
__device__ __forceinline__ void cvt_f2(const uint4 &v, uint32_t &re, uint32_t &im, uint32_t &nim) {
    __half2 r = __floats2half2_rn(__uint_as_float(v.x), __uint_as_float(v.z));
    __half2 i = __floats2half2_rn(__uint_as_float(v.y), __uint_as_float(v.w));
    re = *reinterpret_cast<uint32_t *>(&r);
    im = *reinterpret_cast<uint32_t *>(&i);
    nim = im ^ 0x80008000u;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint4 &v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// byte offset of 16-byte chunk c of row r inside a 128B-swizzled K-major block
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// 8 consecutive spectra [s, s + 8) of one input row as 16 B of complex int8,
// zero-filled outside [0, K) (VEC: the row is 16-byte aligned and s + 8 <= K).
template <bool VEC>
__device__ __forceinline__ uint4 load_i8_chunk(const char2 *row, int s, int K) {
    if (VEC && s + 8 <= K) return __ldg(reinterpret_cast<const uint4 *>(row + s));
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (s + e < K) {
            char2 c = row[s + e];
            uint32_t b = (uint32_t)(uint8_t)c.x | ((uint32_t)(uint8_t)c.y << 8);
            w[e >> 1] |= b << ((e & 1) * 16);
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <bool VEC>
__device__ __forceinline__ uint4 load_f2_pair(const float2 *row, int s, int K) {
    // spectra s, s + 1 as (re0, im0, re1, im1)
    if (VEC && s + 2 <= K) return __ldg(reinterpret_cast<const uint4 *>(row + s));
    float2 a = s < K ? row[s] : make_float2(0.f, 0.f);
    float2 b = s + 1 < K ? row[s + 1] : make_float2(0.f, 0.f);
    return make_uint4(__float_as_uint(a.x), __float_as_uint(a.y), __float_as_uint(b.x), __float_as_uint(b.y));
}

// One pipeline stage of input data held in registers by a producer thread:
// 4 chunks (16 B = 8 spectra of complex int8) of the J block and 4 of the I block.
struct StageRegs {
    uint4 j[4], i[4];
};

template <int MODE, bool VEC>
__global__ void __launch_bounds__(NTHREADS, 1) k_xeng_tc(const XParams p) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char *sgen = smem_raw + (sbase - raw);
    const uint32_t bar0 = sbase + NSTAGE * STAGE_BYTES;
    // barrier layout: full[NSTAGE], empty[NSTAGE], accf[2], acce[2], drain, then tmem addr + abort flag
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NSTAGE + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * NSTAGE + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * NSTAGE + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * NSTAGE + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sgen + NSTAGE * STAGE_BYTES + 8 * (2 * NSTAGE + 5));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            tc::mbar_init(full_bar(s), NPROD);
            tc::mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(accf_bar(b), 1);
            tc::mbar_init(acce_bar(b), NEPI);
        }
        tc::mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nkb = (p.K + KB - 1) / KB;
    // this CTA's items are blockIdx.x + it * gridDim.x; its stages are (it, kb) in order
    const long long my_items = (p.n_items - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const long long n_stages = my_items * nkb;

    if (warp < NPW) {
        // ------------------------------------------------------------ producers
        const int t = threadIdx.x;
        const int c = t & 7;   // 16-byte chunk of a 128-byte fp16 row (8 spectra)
        const int r0 = t >> 3; // first row; rows r0 + 32 q, q < 4
        auto coords = [&](long long n, int &chan, int &I0, int &J0, bool &diag, int &s0) {
            const long long it = n / nkb;
            const int kb = (int)(n - it * nkb);
            int bi, bj;
            decode_item(blockIdx.x + it * gridDim.x, p.n_tiles, chan, bi, bj);
            I0 = bi * TILE;
            J0 = bj * TILE;
            diag = bi == bj;
            s0 = kb * KB;
        };
        if constexpr (MODE == kInt8) {
            auto load = [&](long long n, StageRegs &R) {
                int chan, I0, J0, s0;
                bool diag;
                coords(n, chan, I0, J0, diag, s0);
                const char2 *X = static_cast<const char2 *>(p.X) + (size_t)chan * p.n_in * p.K;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = r0 + 32 * q;
                    const int gj = J0 + r, gi = I0 + r;
                    R.j[q] = gj < p.n_in ? load_i8_chunk<VEC>(X + (size_t)gj * p.K, s0 + 8 * c, p.K)
                                         : make_uint4(0, 0, 0, 0);
                    R.i[q] = (!diag && gi < p.n_in) ? load_i8_chunk<VEC>(X + (size_t)gi * p.K, s0 + 8 * c, p.K)
                                                    : make_uint4(0, 0, 0, 0);
                }
            };
            auto consume = [&](long long n, const StageRegs &R) -> bool {
                const int slot = (int)(n % NSTAGE);
                const uint32_t ph = (uint32_t)((n / NSTAGE) & 1);
                if (!tc::mbar_wait(empty_bar(slot), ph ^ 1u, abort_flag, p.status)) return false;
                int chan, I0, J0, s0;
                bool diag;
                coords(n, chan, I0, J0, diag, s0);
                const uint32_t st = sbase + slot * STAGE_BYTES;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t o = swz(r0 + 32 * q, c);
                    uint4 re, im, nim;
                    cvt_i8(R.j[q], re, im, nim);
                    st_shared_v4(st + OFF_BIM + o, im);
                    st_shared_v4(st + OFF_BRE + o, re);
                    st_shared_v4(st + OFF_BNIM + o, nim);
                    if (!diag) {
                        cvt_i8(R.i[q], re, im, nim);
                        st_shared_v4(st + OFF_ARE + o, re);
                        st_shared_v4(st + OFF_AIM + o, im);
                    }
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(full_bar(slot));
                return true;
            };
            // software pipeline: the loads of stage n + 1 are in flight while stage n is converted
            StageRegs A, Bq;
            if (n_stages > 0) load(0, A);
            for (long long n = 0; n < n_stages; n += 2) {
                if (n + 1 < n_stages) load(n + 1, Bq);
                if (!consume(n, A)) break;
                if (n + 1 >= n_stages) break;
                if (n + 2 < n_stages) load(n + 2, A);
                if (!consume(n + 1, Bq)) break;
            }
        } else {
            for (long long n = 0; n < n_stages; ++n) {
                int chan, I0, J0, s0;
                bool diag;
                coords(n, chan, I0, J0, diag, s0);
                const float2 *X = static_cast<const float2 *>(p.X) + (size_t)chan * p.n_in * p.K;
                // convert to fp16 in registers first (loads in flight before the slot is free)
                uint4 hre[2][4], him[2][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const int g = (side == 0 ? J0 : I0) + r0 + 32 * q;
                        const bool ok = g < p.n_in && (side == 0 || !diag);
                        uint32_t re[4], im[4], nim[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            uint4 v = ok ? load_f2_pair<VEC>(X + (size_t)g * p.K, s0 + 8 * c + 2 * e, p.K)
                                         : make_uint4(0, 0, 0, 0);
                            cvt_f2(v, re[e], im[e], nim[e]);
                        }
                        hre[side][q] = make_uint4(re[0], re[1], re[2], re[3]);
                        him[side][q] = make_uint4(im[0], im[1], im[2], im[3]);
                    }
                }
                const int slot = (int)(n % NSTAGE);
                const uint32_t ph = (uint32_t)((n / NSTAGE) & 1);
                if (!tc::mbar_wait(empty_bar(slot), ph ^ 1u, abort_flag, p.status)) break;
                const uint32_t st = sbase + slot * STAGE_BYTES;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t o = swz(r0 + 32 * q, c);
                    const uint4 M = him[0][q];
                    st_shared_v4(st + OFF_BIM + o, M);
                    st_shared_v4(st + OFF_BRE + o, hre[0][q]);
                    st_shared_v4(st + OFF_BNIM + o,
                                 make_uint4(M.x ^ 0x80008000u, M.y ^ 0x80008000u, M.z ^ 0x80008000u, M.w ^ 0x80008000u));
                    if (!diag) {
                        st_shared_v4(st + OFF_ARE + o, hre[1][q]);
                        st_shared_v4(st + OFF_AIM + o, him[1][q]);
                    }
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(full_bar(slot));
            }
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = tc::idesc_f16(128, 256);
            uint32_t ae_phase[2] = {0, 0};
            long long n = 0;  // stage counter, same sequence as the producers
            bool alive = true;
            for (long long it = 0; it < my_items && alive; ++it) {
                int chan, bi, bj;
                decode_item(blockIdx.x + it * gridDim.x, p.n_tiles, chan, bi, bj);
                const bool diag = bi == bj;
                const int buf = MODE == kInt8 ? 0 : (int)(it & 1);
                const uint32_t d_tmem = tmem + (uint32_t)(buf * 256);
                const int chunk = MODE == kInt8 ? CHUNK_KB : nkb;
                for (int kb = 0; kb < nkb; ++kb, ++n) {
                    const int kin = kb % chunk;
                    if (kin == 0) {
                        // the epilogue has released this accumulator
                        if (!tc::mbar_wait(acce_bar(buf), ae_phase[buf] ^ 1u, abort_flag, p.status)) {
                            alive = false;
                            break;
                        }
                        ae_phase[buf] ^= 1u;
                        tc::tc_fence_after();
                    }
                    const int slot = (int)(n % NSTAGE);
                    if (!tc::mbar_wait(full_bar(slot), (uint32_t)((n / NSTAGE) & 1), abort_flag, p.status)) {
                        alive = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t st = sbase + slot * STAGE_BYTES;
                    const uint32_t a_re = st + (diag ? OFF_BRE : OFF_ARE);
                    const uint32_t a_im = st + (diag ? OFF_BIM : OFF_AIM);
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k) {
                        const uint32_t koff = 32u * k;
                        tc::mma_f16(d_tmem, tc::desc_sw128(a_re + koff), tc::desc_sw128(st + OFF_BRE + koff), IDESC,
                                    (kin > 0 || k > 0) ? 1u : 0u);
                        tc::mma_f16(d_tmem, tc::desc_sw128(a_im + koff), tc::desc_sw128(st + OFF_BIM + koff), IDESC, 1u);
                    }
                    tc::mma_commit(empty_bar(slot));
                    if (kin == chunk - 1 || kb == nkb - 1) tc::mma_commit(accf_bar(buf));
                }
            }
            // drain: every MMA issued must have completed before TMEM is released
            tc::mma_commit(drain_bar);
            tc::mbar_wait(drain_bar, 0u, abort_flag, p.status, 1000000000ull, false);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - (MMA_WARP + 1);  // 0..7
        const int wq = warp & 3;               // TMEM lane quarter this warp may access
        const int h = ew >> 2;                 // column half: j in [64 h, 64 h + 64)
        const int m = wq * 32 + lane;          // tile row = TMEM lane
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t af_phase[2] = {0, 0};
        bool alive = true;
        for (long long it = 0; it < my_items && alive; ++it) {
            int chan, bi, bj;
            decode_item(blockIdx.x + it * gridDim.x, p.n_tiles, chan, bi, bj);
            const int I0 = bi * TILE, J0 = bj * TILE;
            const int i = I0 + m;
            const int buf = MODE == kInt8 ? 0 : (int)(it & 1);
            const uint32_t d_tmem = tmem + lane_off + (uint32_t)(buf * 256);
            if constexpr (MODE == kInt8) {
                const uint32_t r_tmem = tmem + lane_off + 256u;
                const int nch = (nkb + CHUNK_KB - 1) / CHUNK_KB;
                for (int ch = 0; ch < nch; ++ch) {
                    if (!tc::mbar_wait(accf_bar(0), af_phase[0], abort_flag, p.status)) {
                        alive = false;
                        break;
                    }
                    af_phase[0] ^= 1u;
                    tc::tc_fence_after();
#pragma unroll 1
                    for (int cb = 0; cb < 8; ++cb) {
                        // columns: Re 64h + 16 cb (cb < 4), Im 128 + 64h + 16 (cb - 4)
                        const uint32_t col = (uint32_t)((cb < 4 ? 0 : 128) + 64 * h + 16 * (cb & 3));
                        uint32_t d[16], r[16];
                        tc::tmem_ld16(d_tmem + col, d);
                        if (ch > 0) tc::tmem_ld16(r_tmem + col, r);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int x = 0; x < 16; ++x) {
                            int v = __float2int_rn(__uint_as_float(d[x]));
                            r[x] = (uint32_t)((ch > 0 ? (int)r[x] : 0) + v);
                        }
                        tc::tmem_st16(r_tmem + col, r);
                    }
                    tc::tmem_wait_st();
                    tc::tc_fence_before();
                    tc::mbar_arrive(acce_bar(0));
                }
                if (!alive) break;
                // write this tile's INT32 sums (R: Re in columns 0..127, Im in 128..255)
                int2 *acc = static_cast<int2 *>(p.acc) + (size_t)chan * p.B;
#pragma unroll 1
                for (int cb = 0; cb < 4; ++cb) {
                    uint32_t re[16], im[16];
                    const uint32_t col = (uint32_t)(64 * h + 16 * cb);
                    tc::tmem_ld16(r_tmem + col, re);
                    tc::tmem_ld16(r_tmem + 128u + col, im);
                    tc::tmem_wait_ld();
                    if (i < p.n_in) {
                        int2 *row = acc + (size_t)i * (i + 1) / 2;
#pragma unroll
                        for (int x = 0; x < 16; ++x) {
                            const int j = J0 + (int)col + x;
                            if (j <= i) {
                                int2 v = make_int2((int)re[x], (int)im[x]);
                                if (!p.store) {
                                    int2 o = row[j];
                                    v.x += o.x;
                                    v.y += o.y;
                                }
                                row[j] = v;
                            }
                        }
                    }
                }
            } else {
                if (!tc::mbar_wait(accf_bar(buf), af_phase[buf], abort_flag, p.status)) {
                    alive = false;
                    break;
                }
                af_phase[buf] ^= 1u;
                tc::tc_fence_after();
                float2 *acc = static_cast<float2 *>(p.acc) + (size_t)chan * p.B;
                float2 gi = make_float2(1.f, 0.f);
                if (p.gains && i < p.n_in) gi = __ldg(p.gains + i);
#pragma unroll 1
                for (int cb = 0; cb < 4; ++cb) {
                    uint32_t re[16], im[16];
                    const uint32_t col = (uint32_t)(64 * h + 16 * cb);
                    tc::tmem_ld16(d_tmem + col, re);
                    tc::tmem_ld16(d_tmem + 128u + col, im);
                    tc::tmem_wait_ld();
                    if (i < p.n_in) {
                        float2 *row = acc + (size_t)i * (i + 1) / 2;
#pragma unroll
                        for (int x = 0; x < 16; ++x) {
                            const int j = J0 + (int)col + x;
                            if (j <= i) {
                                float2 v = make_float2(__uint_as_float(re[x]), __uint_as_float(im[x]));
                                if (p.gains) {
                                    float2 gj = __ldg(p.gains + j);
                                    float2 w = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
                                    v = make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
                                }
                                if (!p.store) {
                                    float2 o = row[j];
                                    v.x += o.x;
                                    v.y += o.y;
                                }
                                row[j] = v;
                            }
                        }
                    }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(acce_bar(buf));
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == MMA_WARP) tc::tmem_dealloc(tmem, 512);
}

template <int MODE, bool VEC>
corr_status launch_mode(const Handle &h, const void *X, const float2 *gains, bool store, cudaStream_t st) {
    XParams p;
    p.X = X;
    p.acc = h.acc;
    p.gains = gains;
    p.status = h.status;
    p.n_in = h.n_in;
    p.K = h.n_spectra;
    p.nb = (h.n_in + TILE - 1) / TILE;
    p.n_tiles = p.nb * (p.nb + 1) / 2;
    p.B = h.n_base;
    p.n_items = (long long)h.n_chan * p.n_tiles;
    p.store = store ? 1 : 0;
    auto kern = k_xeng_tc<MODE, VEC>;
    CORR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    const long long grid = p.n_items < h.n_sm ? p.n_items : h.n_sm;
    kern<<<(unsigned)grid, NTHREADS, SMEM_BYTES, st>>>(p);
    return check_launch("k_xeng_tc");
}

}  // namespace

corr_status launch_xengine_tc(const Handle &h, const void *chan_in, const float2 *gains, bool store,
                              cudaStream_t st) {
    if (h.precision == CORR_PREC_INT8) {
        const bool vec = (h.n_spectra % 8) == 0;
        return vec ? launch_mode<kInt8, true>(h, chan_in, nullptr, store, st)
                   : launch_mode<kInt8, false>(h, chan_in, nullptr, store, st);
    }
    if (h.precision == CORR_PREC_FP16) {
        const bool vec = (h.n_spectra % 2) == 0;
        return vec ? launch_mode<kFp16, true>(h, chan_in, gains, store, st)
                   : launch_mode<kFp16, false>(h, chan_in, gains, store, st);
    }
    return CORR_EUNSUPPORTED;
}

}  // namespace corr
