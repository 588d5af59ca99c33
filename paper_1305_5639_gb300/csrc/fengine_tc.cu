// Tensor-core F-engine: N = 1024 channels, int8 voltages, 8-bit re-packing into the
// int8 or the planar FP16 layout (no delay compensation, no filter bank; those run on
// the CUDA-core F-engine of fengine_kernel.cuh).
//
// Eq. 1 by the four-step split n = 32 m + t, k = k1 + 32 k2:
//   Y[t][k1]       = sum_m x[32 m + t] W_32^(m k1)      stage 1: 32-point DFTs over m
//   Y'[t][k1]      = Y[t][k1] W_1024^(t k1)              twiddle (CUDA cores, FP32)
//   X[k1 + 32 k2]  = sum_t Y'[t][k1] W_32^(t k2)         stage 2: 32-point DFTs over t
// Both stages are dense contractions of length 32 and run on tcgen05 as real GEMMs
// D = A F^T: the 32-point DFT matrix acting on (Re, Im) pairs is the 64 x 64 real
// matrix F (rows (k, out part), columns (m, in part), K-major), held as FP16
// F = F_h + F_l (to about 2^-22). Stage 1's operand, the int8 samples, is exact in
// FP16: Y = x F_h + x F_l. Stage 2's operand Y' is split the same way on the CUDA
// cores and X = Y'_h F_h + Y'_h F_l + Y'_l F_h (the l l product lies below the FP32
// resolution of the sum). All products accumulate in FP32 in TMEM; the error is a
// few 2^-22 of |X|, within the FP32 FFT's.
//
// One persistent CTA per SM walks work items (one input, 16 consecutive spectra). An
// item is four groups of four frames; a group is one 128-row tile: rows (frame, t) in
// stage 1 and (frame, k1) in stage 2, columns (k, Re / Im) interleaved; the hi/lo
// products of a stage accumulate into the same 64 TMEM columns, and the accumulators
// are four deep, so the MMAs run up to four groups ahead of the drains. Within a
// frame, stage 1's rows are ordered so that the converters' 16-byte stores are free of
// bank conflicts: row 16 e + u holds t = 2 u + e.
// Warp roles:
//   warp 0       issues the MMAs (one thread) and owns the TMEM allocation
//   warps 1-2    convert the raw frames (bulk-copied into a 4-slot ring) into stage 1's
//                A tile, two frames each (one per half warp)
//   warp 3       writes finished items out of the staging rows (corner turn)
//   warps 4-11   drain stage 1, two warps per TMEM lane quarter (16 k1 each): twiddle
//                (held in registers), hi/lo split into stage 2's A tiles
//   warps 12-15  drain stage 2: re-packing into the corner-turn staging rows
// Every hand-over (raw slot, A tiles, TMEM accumulators, staging) is doubled or
// ringed and guarded by mbarriers with bounded waits, so the MMAs of one group overlap
// the drains of its neighbours.
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

#include "internal.h"
#include "requant.cuh"
#include "tc_ptx.cuh"

namespace corr {
namespace {

constexpr int kFtN = 1024, kFtR = 32;  // N = 32 x 32
constexpr int kFtSB = 16;              // spectra per item
constexpr int kFtRoww = kFtSB / 2;     // staging row: 8 words of 16-bit code pairs
constexpr int kFtSw = 2;               // staging swizzle shift: log2(32 / kFtRoww)
constexpr int kFtThreads = 16 * 32;

constexpr int kTileA = 16384;  // 128 rows x 128 B (64 FP16), 128-byte swizzle
constexpr int kTileB = 8192;   // 64 rows x 128 B
constexpr int OFF_A1 = 0;                        // 2 tiles
constexpr int OFF_A2H = OFF_A1 + 2 * kTileA;     // 2 tiles
constexpr int OFF_A2L = OFF_A2H + 2 * kTileA;    // 2 tiles
constexpr int OFF_BH = OFF_A2L + 2 * kTileA;     // F_h
constexpr int OFF_BL = OFF_BH + kTileB;          // F_l
constexpr int OFF_STG = OFF_BL + kTileB;         // 2 staging buffers [k][kFtRoww words]
constexpr int kStgBytes = kFtN * kFtRoww * 4;
constexpr int OFF_RAW = OFF_STG + 2 * kStgBytes; // 4 slots of 4 raw frames (2 KB each)
constexpr int kRawSlot = 4 * 2 * kFtN;
constexpr int OFF_BAR = OFF_RAW + 4 * kRawSlot;
constexpr int kSmemBytes = OFF_BAR + 512 + 1024;  // + alignment slack
static_assert(kSmemBytes <= 232448, "shared memory");

// barrier indices
// (A tiles and staging: 2 deep; TMEM accumulators and raw slots: 4 deep)
constexpr int B_A1F = 0, B_A1E = 2, B_A2F = 4, B_A2E = 6, B_D1F = 8, B_D1E = 12, B_D2F = 16, B_D2E = 20,
              B_SF = 24, B_SE = 26, B_RF = 28, B_RE = 32, B_DONE = 36, kNumBar = 37;

// byte offset of element (row r, column kk) in a K-major tile with 128-byte rows and
// the 128-byte swizzle (8-row groups of 1024 B; 16-byte chunk index XOR row % 8)
__host__ __device__ constexpr uint32_t sw128_off(int r, int kk) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((kk >> 3) ^ (r & 7)) & 7) << 4) + ((kk & 7) << 1));
}

// 16-bit slot of code (k, s) in a staging buffer (word index XOR-swizzled by row)
__device__ __forceinline__ int stg_slot(int k, int s) {
    return k * (2 * kFtRoww) + 2 * ((s >> 1) ^ ((k >> kFtSw) & (kFtRoww - 1))) + (s & 1);
}

// explicit shared-space accesses on 32-bit shared addresses (no generic addressing)
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_u16(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void sts_v4(uint32_t a, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// two complex int8 samples (bytes Re a, Im a, Re b, Im b) -> FP16 pairs (Re a, Im a)
// and (Re b, Im b), exactly: the half with bits 0x64uu is 1024 + u, u the offset-binary
// code q + 128
__device__ __forceinline__ void i8x2_to_h2(uint32_t w, uint32_t &ha, uint32_t &hb) {
    const uint32_t x = w ^ 0x80808080u;
    uint32_t a = __byte_perm(x, 0x64646464u, 0x4140), b = __byte_perm(x, 0x64646464u, 0x4342);
    const __half2 k1152 = __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480));
    __half2 ra = __hsub2(*reinterpret_cast<__half2 *>(&a), k1152);
    __half2 rb = __hsub2(*reinterpret_cast<__half2 *>(&b), k1152);
    ha = *reinterpret_cast<uint32_t *>(&ra);
    hb = *reinterpret_cast<uint32_t *>(&rb);
}

struct FtParams {
    const uint16_t *volt;  // complex int8 samples [n_in][K * 1024]
    const float *scale;    // [1024]
    void *out;             // [1024][PL][n_in][K] 16-bit words
    const float2 *tw;      // [k1][t]
    const uint4 *bimg;     // F_h then F_l, swizzled tile images
    int *status;
    int n_in, K, i0, n_run, vec_out;
};

template <bool PLANAR>
__global__ void __launch_bounds__(kFtThreads, 1) k_fengine_tc(const FtParams p) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw_s = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw_s + 1023u) & ~1023u;
    unsigned char *sg = smem_raw + (sbase - raw_s);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto bar = [&](int b) { return sbase + OFF_BAR + 8u * b; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sg + OFF_BAR + 8 * kNumBar);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int nblk = (p.K + kFtSB - 1) / kFtSB;
    // 32-bit item arithmetic (the host keeps n_run x nblk below 2^28)
    const unsigned n_items = (unsigned)p.n_run * (unsigned)nblk;
    const int my_items = n_items > blockIdx.x ? (int)((n_items - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int total = my_items * 4;  // groups of this CTA
    auto item_of = [&](int r, int &i, int &a0) {
        const unsigned j = blockIdx.x + (unsigned)r * gridDim.x;
        const unsigned ib = j / (unsigned)nblk;
        i = p.i0 + (int)ib;
        a0 = (int)(j - ib * (unsigned)nblk) * kFtSB;
    };

    // ---- set-up: DFT matrices into shared memory; barriers; TMEM
    {
        uint4 *bs = reinterpret_cast<uint4 *>(sg + OFF_BH);
        for (int e = threadIdx.x; e < 2 * kTileB / 16; e += kFtThreads) bs[e] = __ldg(p.bimg + e);
        tc::fence_proxy_async_smem();  // F_h, F_l are read by the tensor cores
    }
    if (threadIdx.x == 0) {
        const int cnt[kNumBar] = {2, 2, 1, 1, 8, 8, 1, 1, 1, 1, 1, 1, 8, 8, 8, 8, 1, 1, 1, 1,
                                  4, 4, 4, 4, 4, 4, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 1};
        for (int b = 0; b < kNumBar; ++b) tc::mbar_init(bar(b), cnt[b]);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;  // D1: columns [0, 256), D2: [256, 512), four buffers of 64 each

    // every lane waits; the warp goes on only if all saw the phase (a timeout in any
    // lane aborts the whole warp, so its control flow stays uniform)
    auto wwait = [&](int b, uint32_t par) {
        const bool ok = tc::mbar_wait(bar(b), par, abort_flag, p.status);
        return __all_sync(0xffffffffu, ok) != 0;
    };

    if (warp == 0) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t ID = tc::idesc_f16(128, 64);
            auto desc = [](uint32_t a) { return tc::desc_sw128(a); };
            const uint32_t bh = sbase + OFF_BH, bl = sbase + OFF_BL;
            // stage 2 trails stage 1 by two groups, so the stage-1 drain has a group of slack
            for (int gs = 0; gs < total + 2; ++gs) {
                if (gs < total) {  // stage 1 of group gs: D1 = x F_h + x F_l
                    const int b = gs & 1, c = gs & 3;
                    if (!tc::mbar_wait(bar(B_A1F + b), (uint32_t)((gs >> 1) & 1), abort_flag, p.status) ||
                        !tc::mbar_wait(bar(B_D1E + c), (uint32_t)(((gs >> 2) & 1) ^ 1), abort_flag, p.status))
                        break;
                    tc::tc_fence_after();
                    const uint32_t d = tmem + 64u * c, a = sbase + OFF_A1 + b * kTileA;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        tc::mma_f16(d, desc(a + 32u * k), desc(bh + 32u * k), ID, k > 0 ? 1u : 0u);
                        tc::mma_f16(d, desc(a + 32u * k), desc(bl + 32u * k), ID, 1u);
                    }
                    tc::mma_commit(bar(B_A1E + b));
                    tc::mma_commit(bar(B_D1F + c));
                }
                if (gs >= 2) {  // stage 2 of group gs - 2: D2 = Y'_h F_h + Y'_h F_l + Y'_l F_h
                    const int g2 = gs - 2, b = g2 & 1, c = g2 & 3;
                    if (!tc::mbar_wait(bar(B_A2F + b), (uint32_t)((g2 >> 1) & 1), abort_flag, p.status) ||
                        !tc::mbar_wait(bar(B_D2E + c), (uint32_t)(((g2 >> 2) & 1) ^ 1), abort_flag, p.status))
                        break;
                    tc::tc_fence_after();
                    const uint32_t d = tmem + 256u + 64u * c;
                    const uint32_t ah = sbase + OFF_A2H + b * kTileA, al = sbase + OFF_A2L + b * kTileA;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        tc::mma_f16(d, desc(ah + 32u * k), desc(bh + 32u * k), ID, k > 0 ? 1u : 0u);
                        tc::mma_f16(d, desc(ah + 32u * k), desc(bl + 32u * k), ID, 1u);
                        tc::mma_f16(d, desc(al + 32u * k), desc(bh + 32u * k), ID, 1u);
                    }
                    tc::mma_commit(bar(B_A2E + b));
                    tc::mma_commit(bar(B_D2F + c));
                }
            }
            // every MMA issued has completed before the TMEM is released
            tc::mma_commit(bar(B_DONE));
            tc::mbar_wait(bar(B_DONE), 0u, abort_flag, p.status, 1000000000ull, false);
        }
        __syncwarp();
    } else if (warp <= 2) {
        // ------------------------------------------------------------ converters
        const int cw = warp - 1;  // frames 2 cw, 2 cw + 1 of the group; lane = t
        const bool issuer = cw == 0 && lane == 0;
        // bulk copy of group gs's frames into raw slot gs % 4 (frames past K are not copied)
        auto issue = [&](int gs) {
            if (gs >= total) return true;
            const int s = (int)(gs & 3);
            if (!tc::mbar_wait(bar(B_RE + s), (uint32_t)(((gs >> 2) & 1) ^ 1), abort_flag, p.status)) return false;
            int i, a0;
            item_of(gs >> 2, i, a0);
            const int a = a0 + 4 * (int)(gs & 3);
            const int nf = max(0, min(4, p.K - a));
            const uint32_t bytes = (uint32_t)nf * 2u * kFtN;
            tc::mbar_arrive_expect_tx(bar(B_RF + s), bytes);
            if (bytes)
                tc::bulk_g2s(sbase + OFF_RAW + s * kRawSlot, p.volt + ((size_t)i * p.K + a) * kFtN, bytes,
                             bar(B_RF + s));
            return true;
        };
        bool alive = true;
        if (issuer)
            for (int gs = 0; gs < 4 && alive; ++gs) alive = issue(gs);
        alive = __shfl_sync(0xffffffffu, alive ? 1 : 0, 0) != 0;
        int i = 0, a0 = 0;  // the current item
        for (int gs = 0; gs < total && alive; ++gs) {
            const int b = gs & 1, s = gs & 3;
            const uint32_t ph = (uint32_t)((gs >> 1) & 1);
            if (!wwait(B_RF + s, (uint32_t)((gs >> 2) & 1)) || !wwait(B_A1E + b, ph ^ 1u)) break;
            if (s == 0) item_of(gs >> 2, i, a0);
            // lanes 0-15 take frame 2 cw, lanes 16-31 frame 2 cw + 1; lane u = lane % 16 owns
            // rows t = 2u, 2u + 1, whose samples share one 32-bit word of each raw row m
            const uint32_t atile = sbase + OFF_A1 + b * kTileA;
            const int q = 2 * cw + (lane >> 4), u = lane & 15;
            const bool valid = a0 + 4 * (gs & 3) + q < p.K;
            const uint32_t rs = sbase + OFF_RAW + s * kRawSlot + q * 2 * kFtN + 4 * u;
            uint32_t w[kFtR];
#pragma unroll
            for (int m = 0; m < kFtR; ++m) w[m] = valid ? lds_u32(rs + 2 * kFtR * m) : 0u;
            // rows of t = 2u and t = 2u + 1 (tile rows 32 q + u and 32 q + 16 + u): columns
            // (m, Re / Im), 16-byte chunks of 4 m
            const int r0 = 32 * q + u;
#pragma unroll
            for (int kc = 0; kc < 8; ++kc) {
                uint4 va, vb;
                i8x2_to_h2(w[4 * kc], va.x, vb.x);
                i8x2_to_h2(w[4 * kc + 1], va.y, vb.y);
                i8x2_to_h2(w[4 * kc + 2], va.z, vb.z);
                i8x2_to_h2(w[4 * kc + 3], va.w, vb.w);
                sts_v4(atile + sw128_off(r0, 8 * kc), va);
                sts_v4(atile + sw128_off(r0 + 16, 8 * kc), vb);
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(bar(B_A1F + b));
                tc::mbar_arrive(bar(B_RE + s));
            }
            if (issuer) alive = issue(gs + 4);
            alive = __shfl_sync(0xffffffffu, alive ? 1 : 0, 0) != 0;
        }
    } else if (warp == 3) {
        // ------------------------------------------------------------ copy-out (corner turn)
        constexpr int PL = PLANAR ? 2 : 1;
        uint16_t *dst = static_cast<uint16_t *>(p.out);
        for (int r = 0; r < my_items; ++r) {
            const int sb = (int)(r & 1);
            if (!wwait(B_SF + sb, (uint32_t)((r >> 1) & 1))) break;
            int i, a0;
            item_of(r, i, a0);
            const int nv = min(kFtSB, p.K - a0);
            const uint32_t stg_s = sbase + OFF_STG + sb * kStgBytes;
            if (nv == kFtSB && p.vec_out) {
                // each lane moves 8 spectra of one channel row: 4 staged words -> one
                // 16-byte store per plane; 16 rows per pass
                const int c8 = lane & 1;
                const size_t dplane = (size_t)p.n_in * p.K / 8;
#pragma unroll 4
                for (int k = lane >> 1; k < kFtN; k += 16) {
                    const int h = (k >> kFtSw) & (kFtRoww - 1);
                    const uint32_t src = stg_s + 4u * (uint32_t)(k * kFtRoww);
                    const uint32_t w0 = lds_u32(src + 4 * ((4 * c8) ^ h)), w1 = lds_u32(src + 4 * ((4 * c8 + 1) ^ h));
                    const uint32_t w2 = lds_u32(src + 4 * ((4 * c8 + 2) ^ h)), w3 = lds_u32(src + 4 * ((4 * c8 + 3) ^ h));
                    uint4 *d = reinterpret_cast<uint4 *>(dst + ((size_t)(PL * k) * p.n_in + i) * p.K + a0 + 8 * c8);
                    if constexpr (PLANAR) {
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
                for (int e = lane; e < kFtN * kFtSB; e += 32) {
                    const int k = e / kFtSB, c = e % kFtSB;
                    if (c < nv) {
                        const uint16_t code = (uint16_t)lds_u16(stg_s + 2 * stg_slot(k, c));
                        uint16_t *row0 = dst + ((size_t)(PL * k) * p.n_in + i) * p.K + a0;
                        if constexpr (PLANAR) {
                            uint32_t re, im;
                            ob_codes_to_f16_planes((uint32_t)code, re, im);
                            row0[c] = (uint16_t)(re & 0xffffu);
                            row0[(size_t)p.n_in * p.K + c] = (uint16_t)(im & 0xffffu);
                        } else {
                            row0[c] = code;
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar(B_SE + sb));
        }
    } else if (warp <= 11) {
        // ------------------------------------------------------------ stage-1 drain
        const int q = warp & 3;                      // TMEM lane quarter = frame of the group
        const int kh = (warp - 4) >> 2;              // k1 in [16 kh, 16 kh + 16)
        const int t = 2 * (lane & 15) + (lane >> 4);  // this lane's row holds t (stage-1 row order)
        float2 tw[16];                               // W_1024^(t k1)
#pragma unroll
        for (int j = 0; j < 16; ++j) tw[j] = __ldg(p.tw + (16 * kh + j) * kFtR + t);
        for (int gs = 0; gs < total; ++gs) {
            const int b = gs & 1, c = gs & 3;
            const uint32_t ph = (uint32_t)((gs >> 1) & 1);
            if (!wwait(B_D1F + c, (uint32_t)((gs >> 2) & 1))) break;
            tc::tc_fence_after();
            // Y: columns 32 kh .. 32 kh + 31 (k1 = 16 kh .. 16 kh + 15, Re / Im)
            uint32_t yh[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 64u * c + 32u * kh, yh);
            tc::tmem_wait_ld();
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar(B_D1E + c));
            // twiddle and hi/lo split, all in registers (yh[2j] <- h, yh[2j + 1] <- l)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float2 y = make_float2(__uint_as_float(yh[2 * j]), __uint_as_float(yh[2 * j + 1]));
                if (kh != 0 || j != 0) y = cmul(y, tw[j]);
                const __half2 h = __floats2half2_rn(y.x, y.y);
                const float2 hf = __half22float2(h);
                const __half2 l = __floats2half2_rn(y.x - hf.x, y.y - hf.y);
                yh[2 * j] = *reinterpret_cast<const uint32_t *>(&h);
                yh[2 * j + 1] = *reinterpret_cast<const uint32_t *>(&l);
            }
            if (!wwait(B_A2E + b, ph ^ 1u)) break;
            const uint32_t ah = sbase + OFF_A2H + b * kTileA, al = sbase + OFF_A2L + b * kTileA;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                // row (q, k1) of stage 2's A tiles, column pair (t, Re / Im)
                const uint32_t off = sw128_off(32 * q + 16 * kh + j, 2 * t);
                sts_u32(ah + off, yh[2 * j]);
                sts_u32(al + off, yh[2 * j + 1]);
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar(B_A2F + b));
        }
    } else {
        // ------------------------------------------------------------ stage-2 drain
        const int q = warp & 3;  // frame of the group; lane = k1
        float sc[kFtR];           // scales of this lane's channels k1 + 32 k2
#pragma unroll
        for (int k2 = 0; k2 < kFtR; ++k2) sc[k2] = __ldg(p.scale + lane + kFtR * k2);
        int i = 0, a0 = 0;  // the current item
        for (int gs = 0; gs < total; ++gs) {
            const int c = gs & 3, g = gs & 3, r = gs >> 2;
            if (g == 0) {
                if (!wwait(B_SE + (r & 1), (uint32_t)(((r >> 1) & 1) ^ 1))) break;
                item_of(r, i, a0);
            }
            if (!wwait(B_D2F + c, (uint32_t)((gs >> 2) & 1))) break;
            tc::tc_fence_after();
            const int s = 4 * g + q;  // spectrum within the item
            const uint32_t stg_s = sbase + OFF_STG + (int)(r & 1) * kStgBytes;
            // X, 16 k2 at a time
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
                uint32_t xa[32];
                tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + 256u + 64u * c + 32u * hlf, xa);
                tc::tmem_wait_ld();
                if (hlf == 1) {
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(bar(B_D2E + c));
                }
                if (a0 + s < p.K) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float2 x = make_float2(__uint_as_float(xa[2 * j]), __uint_as_float(xa[2 * j + 1]));
                        const int k2 = 16 * hlf + j;
                        xa[j] = pack_q<PLANAR>(x, sc[k2]);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) sts_u16(stg_s + 2 * stg_slot(lane + kFtR * (16 * hlf + j), s), xa[j]);
                }
            }
            if (g == 3) {
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(bar(B_SF + (r & 1)));
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

bool fengine_tc_applies(const Handle &h) {
    return h.precision == CORR_PREC_INT8 && h.n_chan == kFtN && !h.dly_int && !h.dly_ph && !h.pfb_win &&
           !(h.flags & CORR_FLAG_FENGINE_CUDACORE) && h.ftc_b != nullptr;
}

// F_h and F_l: the 32-point DFT as a 64 x 64 real matrix, row (k, out part), column
// (m, in part): Re Y += Re x cos + Im x sin, Im Y += -Re x sin + Im x cos (angle
// 2 pi m k / 32), split as F_h = fp16(F), F_l = fp16(F - F_h); stored as the shared-
// memory images of the K-major 128-byte-swizzled operand tiles.
corr_status fengine_tc_init(Handle &h) {
    if (h.precision != CORR_PREC_INT8 || h.n_chan != kFtN) return CORR_OK;
    std::vector<uint16_t> img(2 * kTileB / 2, 0);
    for (int n = 0; n < 64; ++n) {
        const int k = n >> 1, co = n & 1;
        for (int kk = 0; kk < 64; ++kk) {
            const int m = kk >> 1, ci = kk & 1;
            const int j = (m * k) % kFtR;
            const double c = cos2pi(j, kFtR), s = sin2pi(j, kFtR);
            const double v = co == 0 ? (ci == 0 ? c : s) : (ci == 0 ? -s : c);
            const __half hv = __float2half_rn((float)v);
            const __half lv = __float2half_rn((float)(v - (double)__half2float(hv)));
            const uint32_t off = sw128_off(n, kk) / 2;
            img[off] = __half_as_ushort(hv);
            img[kTileB / 2 + off] = __half_as_ushort(lv);
        }
    }
    if (cudaMalloc(&h.ftc_b, 2 * kTileB) != cudaSuccess) {
        cudaGetLastError();
        h.ftc_b = nullptr;
        return CORR_ENOMEM;
    }
    if (cudaMemcpy(h.ftc_b, img.data(), 2 * kTileB, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_cuda_error(cudaGetLastError(), "F-engine DFT matrices");
        return CORR_ECUDA;
    }
    return CORR_OK;
}

corr_status launch_fengine_tc(const Handle &h, const void *volt, const float *scale, void *out, int i0, int n_run,
                              cudaStream_t st) {
    const int n = n_run < 0 ? h.n_in : n_run;
    if (n <= 0) return CORR_OK;
    if (reinterpret_cast<uintptr_t>(volt) % 16 != 0) return CORR_EINVAL;  // bulk copies of whole frames
    FtParams p;
    p.volt = static_cast<const uint16_t *>(volt);
    p.scale = scale;
    p.out = out;
    p.tw = h.twiddle;
    p.bimg = static_cast<const uint4 *>(h.ftc_b);
    p.status = h.status;
    p.n_in = h.n_in;
    p.K = h.n_spectra;
    p.i0 = i0;
    p.n_run = n;
    p.vec_out = (reinterpret_cast<uintptr_t>(out) % 16 == 0) && (h.n_spectra % 8 == 0);
    const long long n_items = (long long)n * ((h.n_spectra + kFtSB - 1) / kFtSB);
    if (n_items >= (1ll << 28)) return CORR_EINVAL;  // 32-bit item arithmetic in the kernel
    const unsigned grid = (unsigned)(n_items < h.n_sm ? n_items : h.n_sm);
    if (h.flags & CORR_FLAG_PLANAR) {
        CORR_CUDA_TRY(cudaFuncSetAttribute(k_fengine_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        k_fengine_tc<true><<<grid, kFtThreads, kSmemBytes, st>>>(p);
    } else {
        CORR_CUDA_TRY(cudaFuncSetAttribute(k_fengine_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        k_fengine_tc<false><<<grid, kFtThreads, kSmemBytes, st>>>(p);
    }
    return check_launch("k_fengine_tc");
}

}  // namespace corr
