// X-engine on tcgen05 tensor cores fed by TMA from the planar FP16 layout
// X[f][plane][input][spectrum] (plane 0 = Re, 1 = Im), Eq. 2 of Section 2 as a
// Hermitian rank-K update V[f] += X[f] X[f]^H over the lower triangle.
//
// For a tile of 128 inputs I (rows) x 128 inputs J, four real MMAs of M = 128,
// N = 128, K = 16 per 16 spectra accumulate
//     D[:, 0:128]   += re_I re_J^T + im_I im_J^T   = Re V_IJ
//     D[:, 128:256] += im_I re_J^T - re_I im_J^T   = Im V_IJ
// the minus sign coming from the instruction descriptor's negate-A bit, so only
// the Re and Im planes are stored. Diagonal tiles (I == J) load the J planes once.
//
// INT8 codes (-128 <= x <= 127) are exact in FP16 and their products exact in
// FP32; each accumulator column sums at most 2 * 128^2 * 512 = 2^24 in magnitude,
// and every integer of magnitude <= 2^24 is an FP32 value, so an FP32 partial
// over <= 512 spectra is an exact integer. The accumulator is double
// buffered in TMEM (2 x 256 columns): while the MMAs fill one buffer with the next
// 512 spectra, the epilogue converts the other exactly and adds it into INT32
// running sums held in registers. The result is bit-exact.
//
// The INT8 and FP16 launches (triangle, rectangle, batched sub-arrays) use the wide
// form instead (the kernel's WIDE variant): two N = 256 MMAs per 16 spectra (six for
// hi/lo), D1 += re_I [re_J; im_J]^T and D2 += im_I [re_J; im_J]^T, with
// Re V = D1a + D2b and Im V = D2a - D1b formed by the epilogue (in INT32 for INT8, in
// FP32 for FP16); it reads 25% fewer operand bytes from shared memory per product (the
// narrow form's limit), and, D1 and D2 filling TMEM, single-buffers the accumulator.
// INT8 folds every 1024 spectra (each half of D1, D2 sums one kind of product). The
// narrow, double-buffered form remains for the short-time INT8 output and the adjoint.
//
// Warp roles (one persistent CTA per SM; 384 threads for the adjoint, 640 otherwise):
//   warp 0       TMA producer (one thread): 3-stage ring of 64-spectrum stages
//   warp 1       TMEM allocator + single-thread MMA issuer
//   warps 4-11   adjoint epilogue, two warps per TMEM lane quarter, each owning half
//                of the tile's columns (wide form and short-time INT8: warps 4-19,
//                four per lane quarter, a quarter of the columns each)
// Every mbarrier wait is bounded; on time-out the CTA records CORR_ETIMEOUT and
// every role leaves its loop.
//
// The same pipeline runs the adjoint's dX GEMM (mode kAdj): Y_f = A_f X_f with
// A_f = 2^e_f G^_f diag(g) (n_in x n_in) and X_f (n_in x K), on rectangular tiles
// (128 rows m of A x 128 spectra a), contracting over the input index j. The J side
// of a stage then comes from a second tensor map holding X_f^T as planes
// [chan][plane][a][j]; per product one N = 256 MMA adds A_re [X_re; X_im]^T to the
// adjacent Re / Im accumulator halves and two N = 128 MMAs add -A_im X_im^T and
// A_im X_re^T, giving exactly Re Y = Ar Xr - Ai Xi and Im Y = Ai Xr + Ar Xi. The
// epilogue scales by 2^-e_f, writes dX = diag(conj g) Y and the partial sums
// sum_a conj(X_ma) Y_ma of dL/dg.
#include <cuda.h>

#include <mutex>
#include <type_traits>

#include "exact_add.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace corr {
namespace {

constexpr int TILE = 128;
constexpr int NSTAGE = 3;
constexpr int NEPI = 256;                 // epilogue threads (warps 4..11)
constexpr int NTHREADS = 384;
constexpr int NTHREADS_WIDE = 640;        // wide INT8 form: 16 epilogue warps (warps 4..19)
constexpr int OSTG_WARP = 4096;           // per epilogue warp: a 32-row slice of the output tile

// Stage geometry. NPL planes per operand side (2: Re, Im; 4: Re_h, Im_h, Re_l, Im_l
// of the hi/lo split); KB spectra per stage: 64 (128-byte rows, 128B swizzle) or
// 32 (64-byte rows, 64B swizzle). A stage holds the NPL planes of the I block
// followed by the NPL planes of the J block.
template <int NPL_, int KB_>
struct TCfg {
    static constexpr int NPL = NPL_;
    static constexpr int KB = KB_;
    static constexpr int PLANE = TILE * KB * 2;
    static constexpr int STAGE_BYTES = 2 * NPL * PLANE;
    static constexpr int CHUNK_KB = 512 / KB;  // INT8: fold every 512 spectra
    static constexpr int OFF_OSTG = NSTAGE * STAGE_BYTES;
    static constexpr int OFF_BAR = OFF_OSTG + 8 * OSTG_WARP;
    static constexpr int SMEM_BYTES = OFF_BAR + 1024 + 256;
    static_assert(SMEM_BYTES <= 232448, "shared memory");
    static __device__ __forceinline__ uint64_t desc(uint32_t a) {
        if constexpr (KB == 64) return tc::desc_sw128(a);
        else return tc::desc_sw64(a);
    }
};

enum Mode { kInt8 = 0, kFp16 = 1, kAdj = 2 };

using SubDesc = BatchSub;

struct TParams {
    void *acc;
    double2 *vis64;  // non-null: integrate straight into the FP64 long-integration buffer
    // batched launch (batch != 0): per-sub tensor maps and descriptors, and each CTA's
    // slice [cta_off[b], cta_off[b + 1]) of the item list (sub, chan, bi | bj << 16)
    const CUtensorMap *tmaps;
    const SubDesc *subs;
    const int4 *items;
    const int *cta_off;
    int batch;
    int c0;  // first channel of a channel-range launch
    const float2 *gains;
    const float *rsc;  // FP16: per-(channel, input) factors 2^-e of the operands' range scaling, or null
    int *status;
    long long B;
    long long n_items;
    int n_in, K, n_tiles, store;
    // adjoint (kAdj): rows = inputs m (n_in), columns = spectra a (n_cols), contraction
    // over j (K = n_in); tiles per channel n_tiles = nbi * nbj
    int adj, nbj, n_cols, tchan0;  // tchan0: channel coordinate origin of the tensor maps
    const float2 *X;               // [chan][m][a] forward input (dg partials)
    float2 *dX;                    // [chan][m][a] or null
    float2 *part;                  // [(chan * nbj + bj) * 2 + half][n_in] or null
    const int *expo;               // [chan - tchan0] power-of-two exponent of A's scaling
    // cross-only rectangle (rect): rows = inputs p0 .. p0 + n_p - 1, columns = inputs
    // q0 .. q0 + n_q - 1 of the same planes; rectangular tiles (nbj column blocks);
    // output [chan][n_p][n_q] (INT32 pairs or float2), overwritten
    int rect, p0, q0, n_p, n_q;
    void *rect_out;
    // short-time visibilities (INT8): every block of st_kb stages (64 spectra each) is
    // also written as [block][chan][plane][B] int32 (plane 0 Re, 1 Im), st_nchan channels
    int *st_out;
    int st_kb, st_nchan;
    // deferred integration dump run by the otherwise idle warps 2 and 3 of every CTA:
    // side_dst[e] += side_src[e] for e < side_n (int2 for INT8, float2 for FP16), each
    // CTA a contiguous slice; side_n = 0: none
    const void *side_src;
    double2 *side_dst;
    long long side_n;
};

// Everything a role needs to know about one work item.
struct Item {
    int chan, bi, bj, n_in, K;
    int cpt, lg_npad, n_chan;  // channel packing: cpt channels of 128 / cpt rows (2^lg_npad) each
    long long B;
    const CUtensorMap *tm;
    void *acc;
};

__device__ __forceinline__ void decode(long long item, int n_tiles, int &chan, int &bi, int &bj);

__device__ __forceinline__ Item get_item(const TParams &p, const CUtensorMap *tmap, long long it) {
    Item r;
    if (p.batch) {
        const int4 e = p.items[p.cta_off[blockIdx.x] + it];
        const SubDesc &sd = p.subs[e.x];
        r.chan = e.y;
        r.bi = e.z & 0xffff;
        r.bj = e.z >> 16;
        r.n_in = sd.n_in;
        r.K = sd.K;
        r.B = sd.B;
        r.tm = p.tmaps + e.x;
        r.acc = sd.acc;
        r.cpt = sd.cpt;
        r.lg_npad = sd.cpt == 1 ? 7 : (sd.cpt == 2 ? 6 : 5);
        r.n_chan = sd.n_chan;
    } else if (p.adj || p.rect) {
        const long long item = blockIdx.x + it * gridDim.x;
        r.chan = (int)(item / p.n_tiles) + p.c0;
        const int t = (int)(item % p.n_tiles);
        r.bi = t / p.nbj;
        r.bj = t % p.nbj;
        r.n_in = p.n_in;
        r.K = p.K;
        r.B = p.B;
        r.tm = tmap;
        r.acc = p.acc;
        r.cpt = 1;
        r.lg_npad = 7;
        r.n_chan = 0x7fffffff;
    } else {
        decode(blockIdx.x + it * gridDim.x, p.n_tiles, r.chan, r.bi, r.bj);
        r.chan += p.c0;
        r.n_in = p.n_in;
        r.K = p.K;
        r.B = p.B;
        r.tm = tmap;
        r.acc = p.acc;
        r.cpt = 1;
        r.lg_npad = 7;
        r.n_chan = 0x7fffffff;
    }
    return r;
}

__device__ __forceinline__ void decode(long long item, int n_tiles, int &chan, int &bi, int &bj) {
    chan = (int)(item / n_tiles);
    int t = (int)(item % n_tiles);
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    bi = r;
    bj = t - r * (r + 1) / 2;
}

// 16-warp epilogues (wide INT8 and short-time INT8): write one warp's INT32 sums of a
// tile (tile rows wq * 32 + lane, tile columns 32 qc .. 32 qc + 31; Re in R[x], Im in
// R[32 + x]) through the warp's 2 KB shared-memory slice, so that consecutive lanes
// write one row's contiguous bytes. Destinations: the packed INT32 accumulator (stored
// or added; packed small sub-arrays map tile rows and columns to (channel, input)
// through lg_npad), the cross-only rectangle, or the FP64 long integration (added).
__device__ __forceinline__ void write_sums16(const int (&R)[64], const Item &itm, const TParams &p,
                                             unsigned char *slice, int wq, int qc, int lane) {
    const int I0 = itm.bi * TILE, J0 = itm.bj * TILE;
    const long long rbase = (long long)itm.chan * itm.B;
    if (p.vis64) {
        // 4 double2 per row slice: 32 rows x 64 B, 4 lanes per row; all reads of a round in
        // flight before its writes
        double2 *sl = reinterpret_cast<double2 *>(slice);
#pragma unroll
        for (int sc = 0; sc < 8; ++sc) {
#pragma unroll
            for (int x = 0; x < 4; ++x)
                sl[lane * 4 + ((x + lane) & 3)] = make_double2((double)R[4 * sc + x], (double)R[32 + 4 * sc + x]);
            __syncwarp();
            double2 o[4];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int r = rr * 8 + (lane >> 2), e = lane & 3;
                const int ii = I0 + wq * 32 + r, jj = J0 + 32 * qc + 4 * sc + e;
                o[rr] = (ii < itm.n_in && jj <= ii) ? __ldcg(p.vis64 + rbase + (long long)ii * (ii + 1) / 2 + jj)
                                                    : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const int r = rr * 8 + (lane >> 2), e = lane & 3;
                const int ii = I0 + wq * 32 + r, jj = J0 + 32 * qc + 4 * sc + e;
                const double2 v = sl[r * 4 + ((e + r) & 3)];
                if (ii < itm.n_in && jj <= ii)
                    p.vis64[rbase + (long long)ii * (ii + 1) / 2 + jj] = make_double2(o[rr].x + v.x, o[rr].y + v.y);
            }
            __syncwarp();
        }
        return;
    }
    int2 *sl = reinterpret_cast<int2 *>(slice);
    int2 *acc = static_cast<int2 *>(itm.acc);
    const int msk = (1 << itm.lg_npad) - 1;
#pragma unroll
    for (int sc = 0; sc < 4; ++sc) {
#pragma unroll
        for (int x = 0; x < 8; ++x) sl[lane * 8 + ((x + lane) & 7)] = make_int2(R[8 * sc + x], R[32 + 8 * sc + x]);
        __syncwarp();
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int r = rr * 4 + (lane >> 3), e = lane & 7;
            const int tr = wq * 32 + r, tcl = 32 * qc + 8 * sc + e;  // tile row / column
            const int q = tr >> itm.lg_npad, qcl = tcl >> itm.lg_npad;
            const int ii = I0 + (tr & msk), jj = J0 + (tcl & msk);
            const int2 v0 = sl[r * 8 + ((e + r) & 7)];
            if (p.rect) {
                // rectangle: tile row ii of group P, column jj of group Q
                if (ii < p.n_p && jj < p.n_q)
                    static_cast<int2 *>(p.rect_out)[((long long)itm.chan * p.n_p + ii) * p.n_q + jj] = v0;
            } else if (q == qcl && itm.chan + q < itm.n_chan && ii < itm.n_in && jj <= ii) {
                int2 *dst = acc + rbase + (long long)q * itm.B + (long long)ii * (ii + 1) / 2 + jj;
                int2 v = v0;
                if (!p.store) {
                    const int2 o = *dst;
                    v.x += o.x;
                    v.y += o.y;
                }
                *dst = v;
            }
        }
        __syncwarp();
    }
}

template <int MODE, class C, bool ST = false, bool WIDE = false>
__global__ void __launch_bounds__((WIDE || (ST && MODE == kInt8)) ? NTHREADS_WIDE : NTHREADS, 1) k_xeng_tma(const __grid_constant__ CUtensorMap tmap,
                                                          const __grid_constant__ CUtensorMap tmapB, const TParams p) {
    constexpr int KB = C::KB, NPL = C::NPL, PLANE = C::PLANE, STAGE_BYTES = C::STAGE_BYTES;
    constexpr int CHUNK_KB = C::CHUNK_KB, OFF_OSTG = C::OFF_OSTG, OFF_BAR = C::OFF_BAR;
    // wide INT8 form: per 16 spectra two N = 256 MMAs, D1 += Re_I [Re_J; Im_J]^T and
    // D2 += Im_I [Re_J; Im_J]^T (the J stage's two planes form one 256-row operand), so
    // each operand tile is read from shared memory once per MMA pair instead of twice;
    // the epilogue forms Re V = D1a + D2b and Im V = D2a - D1b in INT32. Each half of D1,
    // D2 sums one kind of product, |.| <= 128^2 per spectrum, so 1024-spectrum FP32 chunks
    // (|sum| <= 2^24) stay exact; D1 and D2 fill TMEM, so the accumulator is single-buffered.
    constexpr bool W = WIDE && ((MODE == kInt8 && NPL == 2) || MODE == kFp16) && !ST;
    // short-time INT8: the narrow, double-buffered accumulator drained by 16 epilogue
    // warps (warps 4..19), each owning 32 columns of Re V and Im V for 32 rows
    constexpr bool S16 = ST && MODE == kInt8 && NPL == 2 && !WIDE;
    constexpr int CHUNK = W ? 2 * CHUNK_KB : CHUNK_KB;  // INT8 fold period in stages (unused by FP16 and the adjoint)
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    unsigned char *sgen = smem_raw + (sbase - raw);
    const uint32_t bar0 = sbase + OFF_BAR;
    // barriers: full[NSTAGE], empty[NSTAGE], accf[2], acce[2], drain; then tmem slot, abort flag
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (NSTAGE + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (2 * NSTAGE + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (2 * NSTAGE + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (2 * NSTAGE + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sgen + OFF_BAR + 8 * (2 * NSTAGE + 5));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            tc::mbar_init(full_bar(s), 1);
            tc::mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(accf_bar(b), 1);
            tc::mbar_init(acce_bar(b), (W || S16) ? 2 * NEPI : NEPI);
        }
        tc::mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!p.batch) tc::prefetch_tmap(&tmap);
        if constexpr (MODE == kAdj) tc::prefetch_tmap(&tmapB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_u32(tmem_slot), 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long my_items = p.batch ? (long long)(p.cta_off[blockIdx.x + 1] - p.cta_off[blockIdx.x])
                                       : (p.n_items - blockIdx.x + gridDim.x - 1) / gridDim.x;
    // accumulator hand-offs: INT8 one per 512-spectrum chunk, FP16 one per tile

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long n = 0;
            for (long long it = 0; it < my_items; ++it) {
                const Item itm = get_item(p, &tmap, it);
                const int chan = itm.chan - p.tchan0, bi = itm.bi, bj = itm.bj;
                const bool diag = MODE != kAdj && !p.rect && bi == bj;
                // J side: the same planes as the I side, or X^T for the adjoint
                const CUtensorMap *tmj = MODE == kAdj ? &tmapB : itm.tm;
                // first rows of the I and J blocks (the rectangle's groups start at p0, q0)
                const int ri = bi * TILE + (p.rect ? p.p0 : 0), rj = bj * TILE + (p.rect ? p.q0 : 0);
                const int nkb = (itm.K + KB - 1) / KB;
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++n) {
                    const int slot = (int)(n % NSTAGE);
                    if (!tc::mbar_wait(empty_bar(slot), (uint32_t)(((n / NSTAGE) & 1) ^ 1), abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + slot * STAGE_BYTES;
                    const int s0 = kb * KB;
                    if (itm.cpt == 1) {
                        tc::mbar_arrive_expect_tx(full_bar(slot), (diag ? NPL : 2 * NPL) * PLANE);
#pragma unroll
                        for (int pl = 0; pl < NPL; ++pl) {
                            tc::tma_load_4d(st + (NPL + pl) * PLANE, tmj, s0, rj, pl, chan, full_bar(slot));
                            if (!diag) tc::tma_load_4d(st + pl * PLANE, itm.tm, s0, ri, pl, chan, full_bar(slot));
                        }
                    } else {
                        // packed small sub-array: cpt channels stacked in one diagonal tile,
                        // each a box of 128 / cpt rows (the tensor map's box height)
                        const int nv = min(itm.cpt, itm.n_chan - chan);
                        const int npad = 1 << itm.lg_npad;
                        tc::mbar_arrive_expect_tx(full_bar(slot), NPL * nv * npad * KB * 2);
                        for (int q = 0; q < nv; ++q)
#pragma unroll
                            for (int pl = 0; pl < NPL; ++pl)
                                tc::tma_load_4d(st + (NPL + pl) * PLANE + q * npad * KB * 2, itm.tm, s0, 0, pl,
                                                chan + q, full_bar(slot));
                    }
                }
                if (!ok) break;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t ID = tc::idesc_f16(128, 128);
            constexpr uint32_t ID_NEG = tc::idesc_f16(128, 128, /*neg_a=*/true);
            constexpr uint32_t ID256 = tc::idesc_f16(128, 256);
            uint32_t ae_phase[2] = {0, 0};
            long long n = 0, ch = 0;  // stage and accumulator-chunk counters
            bool alive = true;
            for (long long it = 0; it < my_items && alive; ++it) {
                const Item itm = get_item(p, &tmap, it);
                const bool diag = MODE != kAdj && !p.rect && itm.bi == itm.bj;
                const int nkb = (itm.K + KB - 1) / KB;
                const int chunk_kb = MODE == kInt8 ? (ST ? p.st_kb : CHUNK) : nkb;
                uint32_t d_re = 0, d_im = 0;  // wide form: D1 and D2
                int buf = 0;
                for (int kb = 0; kb < nkb; ++kb, ++n) {
                    const int kin = kb % chunk_kb;
                    if (kin == 0) {
                        buf = W ? 0 : (int)(ch & 1);
                        if (!tc::mbar_wait(acce_bar(buf), ae_phase[buf] ^ 1u, abort_flag, p.status)) {
                            alive = false;
                            break;
                        }
                        ae_phase[buf] ^= 1u;
                        tc::tc_fence_after();
                        d_re = tmem + (uint32_t)(buf * 256);
                        d_im = d_re + (W ? 256u : 128u);
                    }
                    const int slot = (int)(n % NSTAGE);
                    if (!tc::mbar_wait(full_bar(slot), (uint32_t)((n / NSTAGE) & 1), abort_flag, p.status)) {
                        alive = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t st = sbase + slot * STAGE_BYTES;
                    const uint32_t a0 = st + (diag ? NPL * PLANE : 0), b0 = st + NPL * PLANE;
                    // complex product of (Re, Im) planes (a, a + PLANE) and (b, b + PLANE):
                    // Re += ar br + ai bi, Im += ai br - ar bi
                    auto cmma = [&](uint32_t a, uint32_t b, uint32_t ko, uint32_t acc) {
                        const uint64_t ar = C::desc(a + ko), ai = C::desc(a + PLANE + ko);
                        const uint64_t br = C::desc(b + ko), bi = C::desc(b + PLANE + ko);
                        tc::mma_f16(d_re, ar, br, ID, acc);
                        tc::mma_f16(d_re, ai, bi, ID, 1u);
                        tc::mma_f16(d_im, ai, br, ID, acc);
                        tc::mma_f16(d_im, ar, bi, ID_NEG, 1u);
                    };
#pragma unroll
                    for (int k = 0; k < KB / 16; ++k) {
                        const uint32_t ko = 32u * k;
                        if constexpr (W) {
                            const uint32_t acc = (kin > 0 || k > 0) ? 1u : 0u;
                            const uint64_t bb = C::desc(b0 + ko);  // [Re_J; Im_J], 256 rows
                            tc::mma_f16(d_re, C::desc(a0 + ko), bb, ID256, acc);
                            tc::mma_f16(d_im, C::desc(a0 + PLANE + ko), bb, ID256, acc);
                            if constexpr (NPL == 4) {
                                // hi/lo: h l and l h into the same accumulators
                                const uint64_t bl = C::desc(b0 + 2 * PLANE + ko);  // [Re_Jl; Im_Jl]
                                tc::mma_f16(d_re, C::desc(a0 + ko), bl, ID256, 1u);
                                tc::mma_f16(d_im, C::desc(a0 + PLANE + ko), bl, ID256, 1u);
                                tc::mma_f16(d_re, C::desc(a0 + 2 * PLANE + ko), bb, ID256, 1u);
                                tc::mma_f16(d_im, C::desc(a0 + 3 * PLANE + ko), bb, ID256, 1u);
                            }
                        } else if constexpr (MODE == kAdj) {
                            // the J side holds X^T's planes (Re, Im, unconjugated), the two
                            // accumulator halves d_re, d_im are adjacent: per product
                            //   [Re Y | Im Y] += A_re [X_re; X_im]^T   (one N = 256 MMA)
                            //   Re Y -= A_im X_im^T,  Im Y += A_im X_re^T
                            // = (A_re X_re - A_im X_im, A_re X_im + A_im X_re): 3 MMAs per
                            // product instead of 4, 7/8 of the operand bytes
                            auto cmma3 = [&](uint32_t a, uint32_t b, uint32_t acc) {
                                tc::mma_f16(d_re, C::desc(a + ko), C::desc(b + ko), ID256, acc);
                                tc::mma_f16(d_re, C::desc(a + PLANE + ko), C::desc(b + PLANE + ko), ID_NEG, 1u);
                                tc::mma_f16(d_im, C::desc(a + PLANE + ko), C::desc(b + ko), ID, 1u);
                            };
                            cmma3(a0, b0, (kin > 0 || k > 0) ? 1u : 0u);  // h h
                            if constexpr (NPL == 4) {
                                cmma3(a0, b0 + 2 * PLANE, 1u);             // h l
                                cmma3(a0 + 2 * PLANE, b0, 1u);             // l h
                            }
                        } else {
                            cmma(a0, b0, ko, (kin > 0 || k > 0) ? 1u : 0u);  // h h
                            if constexpr (NPL == 4) {
                                cmma(a0, b0 + 2 * PLANE, ko, 1u);           // h l
                                cmma(a0 + 2 * PLANE, b0, ko, 1u);           // l h
                            }
                        }
                    }
                    tc::mma_commit(empty_bar(slot));
                    if (kin == chunk_kb - 1 || kb == nkb - 1) {
                        tc::mma_commit(accf_bar(buf));
                        ++ch;
                    }
                }
            }
            tc::mma_commit(drain_bar);
            tc::mbar_wait(drain_bar, 0u, abort_flag, p.status, 1000000000ull, false);
        }
        __syncwarp();
    } else if (W && MODE == kFp16 && warp >= 4) {
        // ------------------------------------------------------------ wide FP16 epilogue
        // 16 warps, four per TMEM lane quarter, each owning columns [32 qc, 32 qc + 32) of
        // Re V = D1a + D2b and Im V = D2a - D1b for its 32 rows (FP32), drained once per
        // tile from the single-buffered accumulator, 8 columns at a time; each piece goes
        // through the warp's 2 KB shared-memory slice so that 8 lanes then write (or
        // read-modify-write) one row's 64 contiguous bytes
        const int ew = warp - 4;               // 0..15
        const int wq = warp & 3;               // TMEM lane quarter this warp may access
        const int qc = ew >> 2;                // column quarter
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        float2 *sl = reinterpret_cast<float2 *>(sgen + OFF_OSTG + ew * (OSTG_WARP / 2));  // [32 rows][8]
        uint32_t af_phase = 0;
        for (long long it = 0; it < my_items; ++it) {
            const Item itm = get_item(p, &tmap, it);
            const int chan = itm.chan;
            const int I0 = itm.bi * TILE, J0 = itm.bj * TILE;
            const int i = I0 + wq * 32 + lane;  // this lane's row while staging
            if (!tc::mbar_wait(accf_bar(0), af_phase, abort_flag, p.status)) break;
            af_phase ^= 1u;
            tc::tc_fence_after();
            const uint32_t d = tmem + lane_off + (uint32_t)(32 * qc);
            // triangle: rows i < n_in, columns j <= i of the packed accumulator (or the FP64
            // buffer); rectangle: rows i < n_p of group P, columns j < n_q of group Q
            const int gi0 = p.rect ? p.p0 : 0, gj0 = p.rect ? p.q0 : 0;
            float2 gi = make_float2(1.f, 0.f);
            if (p.gains && i < (p.rect ? p.n_p : itm.n_in)) gi = __ldg(p.gains + gi0 + i);
            // the operands' range scaling: V_ij carries 2^e_i 2^e_j, undone here (exact)
            const float *rs = p.rsc ? p.rsc + (long long)chan * p.n_in : nullptr;
            float si = 1.f;
            if (rs && i < (p.rect ? p.n_p : itm.n_in)) si = __ldg(rs + gi0 + i);
#pragma unroll 1
            for (int cb = 0; cb < 4; ++cb) {
                // D1 = (re_I re_J | re_I im_J) in columns 0..255, D2 = (im_I re_J | im_I im_J) in 256..511
                uint32_t a1[8], b2[8], a2[8], b1[8];
                tc::tmem_ld8(d + 8u * cb, a1);
                tc::tmem_ld8(d + 384u + 8u * cb, b2);
                tc::tmem_ld8(d + 256u + 8u * cb, a2);
                tc::tmem_ld8(d + 128u + 8u * cb, b1);
                tc::tmem_wait_ld();
                const int jb = J0 + 32 * qc + 8 * cb;  // columns jb .. jb + 7
                // row `lane`, column x at element lane * 8 + ((x + lane / 2) & 7): two
                // wavefronts per 8-byte store of one x and per 4-row read below
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    float2 v = make_float2(__uint_as_float(a1[x]) + __uint_as_float(b2[x]),
                                           __uint_as_float(a2[x]) - __uint_as_float(b1[x]));
                    const int jg = min(jb + x, (p.rect ? p.n_q : itm.n_in) - 1);  // clamped: unused past the end
                    if (rs) {
                        const float sij = si * __ldg(rs + gj0 + jg);
                        v = make_float2(v.x * sij, v.y * sij);
                    }
                    if (p.gains) {
                        const float2 gj = __ldg(p.gains + gj0 + jg);
                        const float2 w = make_float2(gi.x * gj.x + gi.y * gj.y, gi.y * gj.x - gi.x * gj.y);
                        v = make_float2(v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x);
                    }
                    sl[lane * 8 + ((x + (lane >> 1)) & 7)] = v;
                }
                __syncwarp();
                // offsets within the channel's block (below 2^32 entries: one channel's
                // triangle or rectangle)
                float2 val[8];
                uint32_t off[8];
                bool ok[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    const int r = rr * 4 + (lane >> 3), e = lane & 7;
                    const int ii = I0 + wq * 32 + r, jj = jb + e;
                    val[rr] = sl[r * 8 + ((e + (r >> 1)) & 7)];
                    ok[rr] = p.rect ? (ii < p.n_p && jj < p.n_q) : (ii < itm.n_in && jj <= ii);
                    off[rr] = p.rect ? (uint32_t)ii * (uint32_t)p.n_q + jj
                                     : (uint32_t)(((unsigned long long)ii * (unsigned)(ii + 1)) >> 1) + jj;
                }
                __syncwarp();
                // read-modify-writes: every read of a round in flight before its writes
                if (p.vis64) {
                    double2 *dst = p.vis64 + (long long)chan * itm.B;
#pragma unroll
                    for (int h4 = 0; h4 < 8; h4 += 4) {
                        double2 o[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) o[q] = ok[h4 + q] ? __ldcg(dst + off[h4 + q]) : make_double2(0.0, 0.0);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (ok[h4 + q])
                                dst[off[h4 + q]] = add_exact(o[q], val[h4 + q]);  // FP32 sums: conversion in integers
                    }
                } else {
                    float2 *dst = p.rect ? static_cast<float2 *>(p.rect_out) + (long long)chan * p.n_p * p.n_q
                                         : static_cast<float2 *>(itm.acc) + (long long)chan * itm.B;
                    if (!p.store) {
                        float2 o[8];
#pragma unroll
                        for (int rr = 0; rr < 8; ++rr) o[rr] = ok[rr] ? __ldcg(dst + off[rr]) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int rr = 0; rr < 8; ++rr) val[rr] = make_float2(val[rr].x + o[rr].x, val[rr].y + o[rr].y);
                    }
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr)
                        if (ok[rr]) dst[off[rr]] = val[rr];
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(acce_bar(0));
        }
    } else if (W && warp >= 4) {
        // ------------------------------------------------------------ wide INT8 epilogue
        // 16 warps, four per TMEM lane quarter, each owning 32 columns of Re V and Im V:
        // the single-buffered accumulator is drained twice as fast as by 8 warps
        const int ew = warp - 4;               // 0..15
        const int wq = warp & 3;               // TMEM lane quarter this warp may access
        const int qc = ew >> 2;                // column quarter: j in [32 qc, 32 qc + 32)
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t af_phase = 0;
        bool alive = true;
        for (long long it = 0; it < my_items && alive; ++it) {
            const Item itm = get_item(p, &tmap, it);
            const int nkb = (itm.K + KB - 1) / KB;
            const int chunks = (nkb + CHUNK - 1) / CHUNK;
            int R[64];  // INT32 sums: Re of column 32 qc + x in R[x], Im in R[32 + x]
#pragma unroll
            for (int x = 0; x < 64; ++x) R[x] = 0;
            for (int c = 0; c < chunks; ++c) {
                if (!tc::mbar_wait(accf_bar(0), af_phase, abort_flag, p.status)) {
                    alive = false;
                    break;
                }
                af_phase ^= 1u;
                tc::tc_fence_after();
                const uint32_t d = tmem + lane_off + (uint32_t)(32 * qc);
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    // D1 = (ar br | ar bi) in columns 0..255, D2 = (ai br | ai bi) in 256..511
                    uint32_t u[8], w[8];
                    tc::tmem_ld8(d + 8u * cb, u);         // ar br
                    tc::tmem_ld8(d + 384u + 8u * cb, w);  // ai bi
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int x = 0; x < 8; ++x)
                        R[8 * cb + x] += __float2int_rn(__uint_as_float(u[x])) + __float2int_rn(__uint_as_float(w[x]));
                    tc::tmem_ld8(d + 256u + 8u * cb, u);  // ai br
                    tc::tmem_ld8(d + 128u + 8u * cb, w);  // ar bi
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int x = 0; x < 8; ++x)
                        R[32 + 8 * cb + x] += __float2int_rn(__uint_as_float(u[x])) - __float2int_rn(__uint_as_float(w[x]));
                }
                tc::tc_fence_before();
                tc::mbar_arrive(acce_bar(0));
            }
            if (!alive) break;
            write_sums16(R, itm, p, sgen + OFF_OSTG + ew * (OSTG_WARP / 2), wq, qc, lane);
        }
    } else if (S16 && warp >= 4) {
        // ------------------------------------------------------------ short-time INT8 epilogue
        // 16 warps, four per TMEM lane quarter, each owning columns [32 qc, 32 qc + 32) of
        // Re V and Im V for its 32 rows. Every chunk (one short-time block, <= 512 spectra,
        // exact in FP32) is converted, added into the INT32 integration sums and written
        // as the block's visibilities: 16 columns at a time through the warp's 2 KB slice,
        // so that 16 lanes then write one row's 64 contiguous bytes.
        const int ew = warp - 4;               // 0..15
        const int wq = warp & 3;               // TMEM lane quarter this warp may access
        const int qc = ew >> 2;                // column quarter
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        int *sl = reinterpret_cast<int *>(sgen + OFF_OSTG + ew * (OSTG_WARP / 2));  // [32 rows][16]
        uint32_t af_phase[2] = {0, 0};
        long long ch = 0;
        bool alive = true;
        for (long long it = 0; it < my_items && alive; ++it) {
            const Item itm = get_item(p, &tmap, it);
            const int chan = itm.chan;
            const int I0 = itm.bi * TILE, J0 = itm.bj * TILE;
            const int nkb = (itm.K + KB - 1) / KB;
            const int chunks = (nkb + p.st_kb - 1) / p.st_kb;
            // (row offsets ii (ii + 1) / 2 below: one channel's triangle has < 2^32 entries)
            int R[64];  // INT32 sums: Re of j = J0 + 32 qc + x in R[x], Im in R[32 + x]
#pragma unroll
            for (int x = 0; x < 64; ++x) R[x] = 0;
            for (int c = 0; c < chunks; ++c, ++ch) {
                const int buf = (int)(ch & 1);
                if (!tc::mbar_wait(accf_bar(buf), af_phase[buf], abort_flag, p.status)) {
                    alive = false;
                    break;
                }
                af_phase[buf] ^= 1u;
                tc::tc_fence_after();
                const uint32_t d = tmem + lane_off + (uint32_t)(buf * 256) + (uint32_t)(32 * qc);
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    // cb 0, 1: Re columns 32 qc + 16 cb; cb 2, 3: Im columns 128 + 32 qc + 16 (cb - 2),
                    // read from TMEM 8 columns at a time (register budget of 640 threads)
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        uint32_t v[8];
                        tc::tmem_ld8(d + (cb < 2 ? 0u : 128u) + 16u * (cb & 1) + 8u * hf, v);
                        tc::tmem_wait_ld();
                        // row `lane`, column y at word lane * 16 + ((y + lane / 2) & 15): the writes
                        // of one y and the 16-word row reads below are free of bank conflicts
#pragma unroll
                        for (int x = 0; x < 8; ++x) {
                            const int qx = __float2int_rn(__uint_as_float(v[x]));
                            R[16 * cb + 8 * hf + x] += qx;
                            sl[lane * 16 + ((8 * hf + x + (lane >> 1)) & 15)] = qx;
                        }
                    }
                    __syncwarp();
                    const int jb = J0 + 32 * qc + 16 * (cb & 1);
                    int *plane = p.st_out + ((long long)(c * p.st_nchan + chan) * 2 + (cb >> 1)) * itm.B;
#pragma unroll 4
                    for (int rr = 0; rr < 16; ++rr) {
                        const int r = rr * 2 + (lane >> 4), e = lane & 15;
                        const int ii = I0 + wq * 32 + r, jj = jb + e;
                        const uint32_t ro = (uint32_t)(((unsigned long long)ii * (unsigned)(ii + 1)) >> 1);
                        if (ii < itm.n_in && jj <= ii) plane[ro + jj] = sl[r * 16 + ((e + (r >> 1)) & 15)];
                    }
                    __syncwarp();
                }
                tc::tc_fence_before();
                tc::mbar_arrive(acce_bar(buf));
            }
            if (!alive) break;
            write_sums16(R, itm, p, reinterpret_cast<unsigned char *>(sl), wq, qc, lane);
        }
    } else if (MODE == kAdj && warp >= 4) {
        // ------------------------------------------------------------ epilogue (adjoint)
        const int ew = warp - 4;               // 0..7
        const int wq = warp & 3;               // TMEM lane quarter this warp may access
        const int h = ew >> 2;                 // column half: j in [64 h, 64 h + 64)
        const int m = wq * 32 + lane;          // tile row = TMEM lane
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t af_phase[2] = {0, 0};
        long long ch = 0;
        bool alive = true;
        for (long long it = 0; it < my_items && alive; ++it) {
            const Item itm = get_item(p, &tmap, it);
            const int chan = itm.chan;
            const int I0 = itm.bi * TILE, J0 = itm.bj * TILE;
            const int i = I0 + m;
            if constexpr (MODE == kAdj) {
                // dX = conj(g_m) Y and sum_a conj(X_ma) Y_ma over this thread's 64 spectra,
                // Y = 2^-e_f D (rows m = i, columns a = J0 + 64 h + ...)
                const int buf = (int)(ch & 1);
                if (!tc::mbar_wait(accf_bar(buf), af_phase[buf], abort_flag, p.status)) break;
                af_phase[buf] ^= 1u;
                tc::tc_fence_after();
                const uint32_t d = tmem + lane_off + (uint32_t)(buf * 256) + (uint32_t)(64 * h);
                const float sc = ldexpf(1.0f, -__ldg(p.expo + (chan - p.tchan0)));
                float2 gc = make_float2(1.f, 0.f);  // conj(g_m)
                if (p.gains && i < itm.n_in) {
                    const float2 g = __ldg(p.gains + i);
                    gc = make_float2(g.x, -g.y);
                }
                const size_t rowoff = ((size_t)chan * itm.n_in + (size_t)(i < itm.n_in ? i : 0)) * p.n_cols;
                float pr = 0.f, pi = 0.f;
#pragma unroll 1
                for (int cb = 0; cb < 4; ++cb) {
                    uint32_t re[16], im[16];
                    tc::tmem_ld16(d + 16u * cb, re);
                    tc::tmem_ld16(d + 128u + 16u * cb, im);
                    tc::tmem_wait_ld();
                    const int a0 = J0 + 64 * h + 16 * cb;
                    if (a0 + 16 <= p.n_cols) {  // (uniform across the warp)
                        // 16 contiguous spectra: 8 x (two complex values in a float4). X comes in and
                        // dX goes out through the warp's 4 KB slice (row r's float4 x at position
                        // x ^ (r % 8)), so that 8 lanes move each row's 128 contiguous bytes
                        float4 *sl = reinterpret_cast<float4 *>(sgen + OFF_OSTG + ew * OSTG_WARP);
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int r = 4 * k + (lane >> 3), c = lane & 7;  // row of the warp, float4 of the row
                            const int ir = I0 + wq * 32 + r;
                            sl[r * 8 + (c ^ (r & 7))] =
                                ir < itm.n_in
                                    ? __ldg(reinterpret_cast<const float4 *>(p.X + ((size_t)chan * itm.n_in + ir) * p.n_cols + a0) + c)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        __syncwarp();
                        if (i < itm.n_in) {
#pragma unroll
                            for (int x = 0; x < 8; ++x) {
                                float4 &slot = sl[lane * 8 + (x ^ (lane & 7))];
                                const float4 xv = slot;
                                const float y0r = __uint_as_float(re[2 * x]) * sc, y0i = __uint_as_float(im[2 * x]) * sc;
                                const float y1r = __uint_as_float(re[2 * x + 1]) * sc, y1i = __uint_as_float(im[2 * x + 1]) * sc;
                                pr += xv.x * y0r + xv.y * y0i + xv.z * y1r + xv.w * y1i;
                                pi += xv.x * y0i - xv.y * y0r + xv.z * y1i - xv.w * y1r;
                                slot = make_float4(gc.x * y0r - gc.y * y0i, gc.x * y0i + gc.y * y0r,
                                                   gc.x * y1r - gc.y * y1i, gc.x * y1i + gc.y * y1r);
                            }
                        }
                        __syncwarp();
                        if (p.dX) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const int r = 4 * k + (lane >> 3), c = lane & 7;
                                const int ir = I0 + wq * 32 + r;
                                if (ir < itm.n_in)
                                    reinterpret_cast<float4 *>(p.dX + ((size_t)chan * itm.n_in + ir) * p.n_cols + a0)[c] =
                                        sl[r * 8 + (c ^ (r & 7))];
                            }
                        }
                        __syncwarp();
                    } else if (i < itm.n_in) {
#pragma unroll 1
                        for (int x = 0; x < 16; ++x) {
                            if (a0 + x >= p.n_cols) break;
                            const float2 xv = __ldg(p.X + rowoff + a0 + x);
                            const float yr = __uint_as_float(re[x]) * sc, yi = __uint_as_float(im[x]) * sc;
                            pr += xv.x * yr + xv.y * yi;
                            pi += xv.x * yi - xv.y * yr;
                            if (p.dX) p.dX[rowoff + a0 + x] = make_float2(gc.x * yr - gc.y * yi, gc.x * yi + gc.y * yr);
                        }
                    }
                }
                tc::tc_fence_before();
                tc::mbar_arrive(acce_bar(buf));
                ++ch;
                if (p.part && i < itm.n_in)
                    p.part[((size_t)chan * p.nbj + itm.bj) * 2 * itm.n_in + (size_t)h * itm.n_in + i] = make_float2(pr, pi);
            }
        }
    }

    if ((warp == 2 || warp == 3) && p.side_n > 0) {
        // ------------------------------------------------------------ deferred dump
        // The previous integration's accumulator into the FP64 long integration, in this
        // CTA's slice, while the other roles run the X-engine: loads of 8 elements per
        // thread in flight before their stores. The sums are exact (integer values below
        // 2^53 for INT8; the FP64 add of the FP32 sums for FP16, as the dump kernel).
        using AccT = typename std::conditional<MODE == kInt8, int2, float2>::type;
        const AccT *src = static_cast<const AccT *>(p.side_src);
        const long long lo = p.side_n * blockIdx.x / gridDim.x, hi = p.side_n * (blockIdx.x + 1) / gridDim.x;
        constexpr int U = 8;
        constexpr long long BATCH = 64 * U;  // elements per round of the 64 threads
        constexpr int AHEAD = 4;              // rounds prefetched into L2 ahead of the loads
        const int lt = threadIdx.x - 64;  // 0 .. 63
        // bulk L2 prefetch of rounds [r0, r1) of both streams (one thread; 16-byte aligned
        // ranges inside the buffers), so that the loads below hit L2
        auto prefetch = [&](long long e_begin, long long e_end) {
            e_begin = max(e_begin, lo);
            e_end = min(e_end, hi);
            if (e_end <= e_begin) return;
            const uintptr_t sa = reinterpret_cast<uintptr_t>(src + e_begin) & ~(uintptr_t)15;
            const uintptr_t se = reinterpret_cast<uintptr_t>(src + e_end) & ~(uintptr_t)15;
            const uintptr_t da = reinterpret_cast<uintptr_t>(p.side_dst + e_begin);
            const uintptr_t de = reinterpret_cast<uintptr_t>(p.side_dst + e_end);
            if (se > sa) tc::prefetch_l2_bulk(reinterpret_cast<const void *>(sa), (uint32_t)(se - sa));
            tc::prefetch_l2_bulk(reinterpret_cast<const void *>(da), (uint32_t)(de - da));
        };
        if (lt == 0) prefetch(lo, lo + AHEAD * BATCH);
        for (long long e0 = lo + lt; e0 < hi; e0 += BATCH) {
            if (*abort_flag) break;
            if (lt == 0) prefetch(e0 + AHEAD * BATCH, e0 + (AHEAD + 1) * BATCH);
            AccT a[U];
            double2 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long e = e0 + 64 * u;
                if (e < hi) {
                    a[u] = __ldcs(src + e);
                    v[u] = __ldcg(p.side_dst + e);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long e = e0 + 64 * u;
                if (e < hi) p.side_dst[e] = make_double2(v[u].x + (double)a[u].x, v[u].y + (double)a[u].y);
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------ tensor map
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

}  // namespace

bool tma_available() { return encode_fn() != nullptr; }

bool xengine_tma_supported(const Handle &h) { return (h.n_spectra % 8) == 0 && encode_fn() != nullptr; }

corr_status tma_encode_planar(void *tmap128, const void *planes, int n_in, int n_chan, int K, int npl,
                              int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error_text("cuTensorMapEncodeTiled is not available from the driver");
        return CORR_EUNSUPPORTED;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)n_in, (cuuint64_t)npl, (cuuint64_t)n_chan};
    const cuuint64_t strides[3] = {(cuuint64_t)K * 2, (cuuint64_t)K * 2 * n_in, (cuuint64_t)K * 2 * n_in * npl};
    const cuuint32_t box[4] = {64, (cuuint32_t)box_rows, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(static_cast<CUtensorMap *>(tmap128), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(planes),
                     dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error_text("cuTensorMapEncodeTiled rejected a planar layout");
        return CORR_EINVAL;
    }
    return CORR_OK;
}

// Every INT8 launch but the short-time one: the wide form, 640 threads.
corr_status launch_int8_wide(const CUtensorMap &tmap, const TParams &p, unsigned grid, cudaStream_t st) {
    using C = TCfg<2, 64>;
    auto kern = k_xeng_tma<kInt8, C, false, true>;
    CORR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
    kern<<<grid, NTHREADS_WIDE, C::SMEM_BYTES, st>>>(tmap, tmap, p);
    return CORR_OK;
}

// FP16 and hi/lo launches (triangle, rectangle): the wide form, 640 threads.
corr_status launch_fp16_wide(const CUtensorMap &tmap, const TParams &p, int npl, unsigned grid, cudaStream_t st) {
    if (npl == 2) {
        using C = TCfg<2, 64>;
        auto kern = k_xeng_tma<kFp16, C, false, true>;
        CORR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
        kern<<<grid, NTHREADS_WIDE, C::SMEM_BYTES, st>>>(tmap, tmap, p);
    } else {
        using C = TCfg<4, 32>;
        auto kern = k_xeng_tma<kFp16, C, false, true>;
        CORR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
        kern<<<grid, NTHREADS_WIDE, C::SMEM_BYTES, st>>>(tmap, tmap, p);
    }
    return CORR_OK;
}

corr_status launch_xengine_tma_batch(const void *d_tmaps, const BatchSub *d_subs, const int4 *d_items,
                                     const int *d_cta_off, int grid, int *status, cudaStream_t st) {
    TParams p{};
    p.tmaps = static_cast<const CUtensorMap *>(d_tmaps);
    p.subs = d_subs;
    p.items = d_items;
    p.cta_off = d_cta_off;
    p.batch = 1;
    p.status = status;
    p.store = 1;
    CUtensorMap dummy{};  // unused in batched mode (each item names its sub's map)
    const corr_status s = launch_int8_wide(dummy, p, (unsigned)grid, st);
    if (s != CORR_OK) return s;
    return check_launch("k_xeng_tma (batched)");
}

corr_status launch_xengine_tma(const Handle &h, const void *planes, int npl, const float2 *gains,
                               const float *row_scale, int kstride, bool store, cudaStream_t st) {
    return launch_xengine_tma_range(h, planes, npl, gains, row_scale, kstride, store, 0, h.n_chan, st);
}

corr_status launch_xengine_tma_range(const Handle &h, const void *planes, int npl, const float2 *gains,
                                     const float *row_scale, int kstride, bool store, int c0, int c1,
                                     cudaStream_t st) {
    if (c1 <= c0) return CORR_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error_text("cuTensorMapEncodeTiled is not available from the driver");
        return CORR_EUNSUPPORTED;
    }
    if ((kstride % 8) != 0 || kstride < h.n_spectra || (npl != 2 && npl != 4)) return CORR_EUNSUPPORTED;
    const int kb = npl == 2 ? 64 : 32;
    // planar FP16 tensor: dims (innermost first) spectrum, input, plane, channel; rows of
    // kstride elements (16-byte multiples), spectra past n_spectra read as zeros
    CUtensorMap tmap;
    const cuuint64_t dims[4] = {(cuuint64_t)h.n_spectra, (cuuint64_t)h.n_in, (cuuint64_t)npl, (cuuint64_t)h.n_chan};
    const cuuint64_t strides[3] = {(cuuint64_t)kstride * 2, (cuuint64_t)kstride * 2 * h.n_in,
                                   (cuuint64_t)kstride * 2 * h.n_in * npl};
    const cuuint32_t box[4] = {(cuuint32_t)kb, TILE, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(planes), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, kb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error_text("cuTensorMapEncodeTiled rejected the planar layout");
        return CORR_EINVAL;
    }
    TParams p{};
    p.acc = h.acc;
    p.vis64 = (h.flags & CORR_FLAG_FUSED_DUMP) ? h.vis64 : nullptr;
    p.gains = gains;
    p.rsc = row_scale;
    if (h.dump_pending) {
        // the previous integration's deferred dump rides along (all channels, one launch)
        p.side_dst = h.vis64;
        p.side_src = h.pending_src;
        p.side_n = (long long)h.n_chan * h.n_base;
    }
    p.status = h.status;
    p.B = h.n_base;
    const int nb = (h.n_in + TILE - 1) / TILE;
    p.n_tiles = nb * (nb + 1) / 2;
    p.n_items = (long long)(c1 - c0) * p.n_tiles;
    p.c0 = c0;
    p.n_in = h.n_in;
    p.K = h.n_spectra;
    p.store = store ? 1 : 0;
    if (h.precision == CORR_PREC_INT8 && h.st_out) {
        p.st_out = h.st_out;
        p.st_kb = h.st_block / 64;
        p.st_nchan = h.n_chan;
    }
    const unsigned grid = (unsigned)(p.n_items < h.n_sm ? p.n_items : h.n_sm);
    StageScope sc(h, CORR_STAGE_XENGINE, st);
    if (h.precision == CORR_PREC_INT8 && p.st_out) {
        using C = TCfg<2, 64>;
        auto kern = k_xeng_tma<kInt8, C, true>;
        CORR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
        kern<<<grid, NTHREADS_WIDE, C::SMEM_BYTES, st>>>(tmap, tmap, p);
    } else if (h.precision == CORR_PREC_INT8) {
        const corr_status s = launch_int8_wide(tmap, p, grid, st);
        if (s != CORR_OK) return s;
    } else {
        const corr_status s = launch_fp16_wide(tmap, p, npl, grid, st);
        if (s != CORR_OK) return s;
    }
    return check_launch("k_xeng_tma");
}

corr_status launch_xengine_tma_rect(const Handle &h, const void *planes, int npl, const float2 *gains,
                                    const float *row_scale, int kstride, int p0, int n_p, int q0, int n_q, void *out,
                                    cudaStream_t st) {
    if (n_p <= 0 || n_q <= 0) return CORR_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error_text("cuTensorMapEncodeTiled is not available from the driver");
        return CORR_EUNSUPPORTED;
    }
    if ((kstride % 8) != 0 || kstride < h.n_spectra || (npl != 2 && npl != 4)) return CORR_EUNSUPPORTED;
    const int kb = npl == 2 ? 64 : 32;
    CUtensorMap tmap;
    const cuuint64_t dims[4] = {(cuuint64_t)h.n_spectra, (cuuint64_t)h.n_in, (cuuint64_t)npl, (cuuint64_t)h.n_chan};
    const cuuint64_t strides[3] = {(cuuint64_t)kstride * 2, (cuuint64_t)kstride * 2 * h.n_in,
                                   (cuuint64_t)kstride * 2 * h.n_in * npl};
    const cuuint32_t box[4] = {(cuuint32_t)kb, TILE, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(planes), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, kb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error_text("cuTensorMapEncodeTiled rejected the planar layout");
        return CORR_EINVAL;
    }
    TParams p{};
    p.gains = gains;
    p.rsc = row_scale;
    p.status = h.status;
    p.B = h.n_base;
    p.rect = 1;
    p.p0 = p0;
    p.q0 = q0;
    p.n_p = n_p;
    p.n_q = n_q;
    p.rect_out = out;
    const int nbi = (n_p + TILE - 1) / TILE;
    p.nbj = (n_q + TILE - 1) / TILE;
    p.n_tiles = nbi * p.nbj;
    p.n_items = (long long)h.n_chan * p.n_tiles;
    p.n_in = h.n_in;
    p.K = h.n_spectra;
    p.store = 1;
    const unsigned grid = (unsigned)(p.n_items < h.n_sm ? p.n_items : h.n_sm);
    StageScope sc(h, CORR_STAGE_XENGINE, st);
    if (h.precision == CORR_PREC_INT8) {
        const corr_status s = launch_int8_wide(tmap, p, grid, st);
        if (s != CORR_OK) return s;
    } else {
        const corr_status s = launch_fp16_wide(tmap, p, npl, grid, st);
        if (s != CORR_OK) return s;
    }
    return check_launch("k_xeng_tma (rectangle)");
}

// Planar FP16 operand tensor [chan][plane][rows][cols] (cols innermost) with a box
// of kb columns x 128 rows.
static corr_status encode_planes(CUtensorMap *tm, const void *planes, int cols, int rows, int npl, int n_chan,
                                 int kb) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error_text("cuTensorMapEncodeTiled is not available from the driver");
        return CORR_EUNSUPPORTED;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)npl, (cuuint64_t)n_chan};
    const cuuint64_t strides[3] = {(cuuint64_t)cols * 2, (cuuint64_t)cols * 2 * rows,
                                   (cuuint64_t)cols * 2 * rows * npl};
    const cuuint32_t box[4] = {(cuuint32_t)kb, TILE, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(planes), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, kb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error_text("cuTensorMapEncodeTiled rejected an operand layout");
        return CORR_EINVAL;
    }
    return CORR_OK;
}

corr_status launch_adjoint_tma(const Handle &h, const void *a_planes, const void *b_planes, const int *expo,
                               const float2 *X, const float2 *gains, float2 *dX, float2 *part, int c0, int c1,
                               cudaStream_t st) {
    if (c1 <= c0) return CORR_OK;
    if ((h.n_in % 8) != 0) return CORR_EUNSUPPORTED;
    using C = TCfg<4, 32>;
    const int cb = c1 - c0;
    CUtensorMap ta, tb;
    corr_status s = encode_planes(&ta, a_planes, h.n_in, h.n_in, 4, cb, C::KB);
    if (s != CORR_OK) return s;
    s = encode_planes(&tb, b_planes, h.n_in, h.n_spectra, 4, cb, C::KB);
    if (s != CORR_OK) return s;
    TParams p{};
    p.gains = gains;
    p.status = h.status;
    p.adj = 1;
    p.n_in = h.n_in;
    p.K = h.n_in;  // contraction over the input index j
    p.n_cols = h.n_spectra;
    const int nbi = (h.n_in + TILE - 1) / TILE;
    p.nbj = (h.n_spectra + TILE - 1) / TILE;
    p.n_tiles = nbi * p.nbj;
    p.n_items = (long long)cb * p.n_tiles;
    p.c0 = c0;
    p.tchan0 = c0;
    p.X = X;
    p.dX = dX;
    p.part = part;
    p.expo = expo;
    const unsigned grid = (unsigned)(p.n_items < h.n_sm ? p.n_items : h.n_sm);
    StageScope sc(h, CORR_STAGE_ADJ_GEMM, st);
    CORR_CUDA_TRY(cudaFuncSetAttribute(k_xeng_tma<kAdj, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
    k_xeng_tma<kAdj, C><<<grid, NTHREADS, C::SMEM_BYTES, st>>>(ta, tb, p);
    return check_launch("k_xeng_tma (adjoint)");
}

}  // namespace corr
