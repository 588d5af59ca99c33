// Internal declarations shared by the libcorr translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "corr.h"

namespace corr {

// Optional per-stage timing of the kernels a handle launches (corr_set_stage_timing):
// a pair of CUDA events around each stage's launches on the stream they run on.
struct StageClock {
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;  // spare events (created on demand, kept for reuse)
    std::vector<Rec> recs;          // recorded, not yet read
    int64_t launches[CORR_STAGE_COUNT] = {};
    bool on = false;
    bool overflow = false;          // more records than kMaxRecs since the last read
    static constexpr size_t kMaxRecs = 1 << 16;
};

// Handle state. Device buffers are owned by the library.
struct Handle {
    int32_t n_ant, n_pol, n_in, n_chan, n_spectra;
    int64_t n_base;  // B = n_in (n_in + 1) / 2
    int32_t precision, xengine, flags;
    int32_t device;
    int32_t n_sm;
    // integration accumulator [n_chan][B]: int2 (INT8) or float2 (float paths)
    void *acc = nullptr;
    bool acc_zero = true;        // accumulator known to be all-zero (X-engine may store instead of add)
    // deferred dump (tensor-core X-engine): corr_dump without a copy swaps acc with
    // acc_alt and leaves the finished integration in pending_src; the next X-engine
    // launch adds it to vis64 from idle warps (or a flush runs the dump kernel)
    void *acc_alt = nullptr;
    bool dump_pending = false;
    const void *pending_src = nullptr;
    int64_t acc_spectra = 0;     // spectra accumulated since the last dump (INT8 overflow guard)
    double2 *vis64 = nullptr;    // FP64 long-integration buffer [n_chan][B]
    float2 *twiddle = nullptr;   // F-engine twiddles W_N^(t k1), [k1][t], N = T1 x T2
    void *ftc_b = nullptr;       // tensor-core F-engine DFT matrices F_h, F_l (N = 1024, INT8)
    int32_t *dly_int = nullptr;  // delay compensation (null: off): integer advance per input
    float2 *dly_ph = nullptr;    //   and phase tables [n_in][T1 + T2]: exp(+j 2 pi k1 f / N), exp(+j 2 pi T1 k2 f / N)
    float *pfb_win = nullptr;    // polyphase filter-bank window [pfb_taps][n_chan] (null: off)
    int32_t pfb_taps = 0;
    void *pfb_y = nullptr;       //   its FIR output, complex FP32 [n_in][n_spectra][n_chan]
    int32_t *st_out = nullptr;   // short-time visibilities (caller's buffer; null: off)
    int32_t st_block = 0;        //   spectra per block
    int32_t *status = nullptr;   // device status word (0 ok, else CORR_* code set by a kernel)
    double *power64 = nullptr;   // [n_chan] scratch for corr_fengine_power
    void *planar_ws = nullptr;   // FP16 operand planes for the FP16 tensor-core paths (first use)
    size_t planar_ws_bytes = 0;
    float2 *bwd_ws = nullptr;    // corr_backward workspace (dg partials; tensor-core operand planes)
    cudaStream_t bwd_side = nullptr;  // tensor-core backward: side stream for the operand passes
    cudaEvent_t bwd_ev[5] = {};       //   and its events
    // host-buffer pipeline (corr_fx_host): two device copies of the inputs (calls use
    // them in turn), the channelised data, two copy streams and per-block events (first use)
    void *fx_volt[2] = {nullptr, nullptr}, *fx_chan = nullptr;
    int fx_par = 0;  // the input copy the next call fills
    cudaStream_t fx_in = nullptr, fx_out = nullptr;
    cudaEvent_t fx_ev[40] = {};
    bool fx_ready = false;  // every fx_* resource above was created
    size_t bwd_ws_bytes = 0;
    StageClock *clock = nullptr;  // stage timing (null until first enabled)
};

// Records the stage's start event on construction and its end event on destruction
// when the handle's stage timing is on; counts n_launch kernel launches either way.
class StageScope {
  public:
    StageScope(const Handle &h, int stage, cudaStream_t st, int n_launch = 1);
    ~StageScope();
    StageScope(const StageScope &) = delete;
    StageScope &operator=(const StageScope &) = delete;

  private:
    StageClock *c_;
    int stage_;
    cudaStream_t st_;
    cudaEvent_t a_ = nullptr;
};

// Error bookkeeping (per thread).
void set_cuda_error(cudaError_t e, const char *what);
void set_error_text(const char *text);
corr_status check_launch(const char *what);

#define CORR_CUDA_TRY(expr)                                  \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) {                             \
            ::corr::set_cuda_error(_e, #expr);               \
            return CORR_ECUDA;                               \
        }                                                    \
    } while (0)

// Makes a device current for the lifetime of the guard and restores the previous one.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// Kernel launchers (return CORR_OK or an error status).
corr_status launch_fengine(const Handle &h, const void *volt, const float *scale, void *out,
                           cudaStream_t st);
corr_status launch_fengine_power(const Handle &h, const void *volt, float *power, cudaStream_t st);
corr_status launch_xengine_cudacore(const Handle &h, const void *chan_in, const float2 *gains,
                                    bool store, cudaStream_t st);
corr_status launch_dump(const Handle &h, cudaStream_t st);
corr_status launch_dump_range(const Handle &h, int c0, int c1, cudaStream_t st);
// The dump of an accumulator other than the handle's current one (a deferred dump).
corr_status launch_dump_src(const Handle &h, const void *acc, cudaStream_t st);
corr_status launch_fengine_range(const Handle &h, const void *volt, const float *scale, void *out, int i0, int n_run,
                                 cudaStream_t st);
// TMA X-engine over channels [c0, c1) of planar FP16 operands [chan][npl][n_in][kstride]
// (kstride >= n_spectra, a multiple of 8); row_scale [chan][n_in] (or null): the
// factors 2^-e of the FP16 paths' per-row range scaling, undone in the epilogue.
corr_status launch_xengine_tma_range(const Handle &h, const void *planes, int npl, const float2 *gains,
                                     const float *row_scale, int kstride, bool store, int c0, int c1,
                                     cudaStream_t st);
size_t backward_workspace_bytes(const Handle &h);
corr_status launch_backward_ws(const Handle &h, const float2 *grad_vis, const float2 *chan_in,
                               const float2 *gains, float2 *grad_chan, float2 *grad_gains, float2 *ws,
                               cudaStream_t st);
// Tensor-core adjoint (FP16 hi/lo): workspace bytes and channel-block size, the
// whole backward pass, and its dX GEMM (see adjoint_tc.cu, xengine_tma.cu).
size_t backward_tc_workspace_bytes(const Handle &h, int *chan_block);
corr_status launch_backward_tc(const Handle &h, const float2 *grad_vis, const float2 *chan_in, const float2 *gains,
                               float2 *grad_chan, float2 *grad_gains, void *ws, cudaStream_t st,
                               cudaStream_t side, cudaEvent_t *ev);
corr_status launch_adjoint_tma(const Handle &h, const void *a_planes, const void *b_planes, const int *expo,
                               const float2 *X, const float2 *gains, float2 *dX, float2 *part, int c0, int c1,
                               cudaStream_t st);
// dL/dg from per-row partials part[p][n_in], p < n_part, summed in a fixed order
// (scratch: adj_reduce_scratch_bytes(n_in) bytes, 16-byte aligned).
size_t adj_reduce_scratch_bytes(int n_in);
inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
corr_status launch_adj_reduce(const float2 *part, double2 *scratch, float2 *dg, int n_in, long long n_part,
                              cudaStream_t st);
// Cross-only rectangle of the visibility matrix on the TMA X-engine: inputs
// [p0, p0 + n_p) x [q0, q0 + n_q), output [n_chan][n_p][n_q] overwritten.
corr_status launch_xengine_tma_rect(const Handle &h, const void *planes, int npl, const float2 *gains,
                                    const float *row_scale, int kstride, int p0, int n_p, int q0, int n_q, void *out,
                                    cudaStream_t st);
// Bounded-wait self-test (selftest.cu): CORR_OK if a wait that nothing completes gave up
// after limit_ns, recorded CORR_ETIMEOUT and returned.
corr_status selftest_bounded_wait(uint64_t limit_ns);

// Polyphase filter bank: FIR pass of inputs [i0, i0 + n_run) into h.pfb_y (pfb.cu).
corr_status launch_pfb_fir(const Handle &h, const void *volt, int i0, int n_run, cudaStream_t st);
bool fengine_supported(int n_chan);
// tensor-core F-engine (fengine_tc.cu): N = 1024, INT8, no delays or filter bank
bool fengine_tc_applies(const Handle &h);
corr_status fengine_tc_init(Handle &h);
corr_status launch_fengine_tc(const Handle &h, const void *volt, const float *scale, void *out, int i0, int n_run,
                              cudaStream_t st);
bool xengine_tma_supported(const Handle &h);
corr_status launch_xengine_tma(const Handle &h, const void *planes, int npl, const float2 *gains,
                               const float *row_scale, int kstride, bool store, cudaStream_t st);
// FP16 operand preparation (prep.cu): complex float [chan][n_in][K] -> planes
// [chan][npl][n_in][planar_kstride(K)] with a per-row power-of-two range scale, whose
// reciprocals planar_row_scale() points at, inside one workspace of planar_ws_bytes().
int planar_kstride(int K);
size_t planar_ws_bytes(const Handle &h, int npl);
float *planar_row_scale(const Handle &h, void *ws, int npl);
corr_status launch_to_planar(const Handle &h, const float2 *X, void *ws, int npl, cudaStream_t st);
// Complex int8 [chan][n_in][K] -> planar FP16 codes [chan][2][n_in][planar_kstride(K)] (exact).
corr_status launch_i8_to_planar(const Handle &h, const void *X, void *ws, cudaStream_t st);
bool tma_available();

// One sub-array of a batched X-engine launch (device-side descriptor).
struct BatchSub {
    void *acc;    // INT32 pairs [n_chan][B] (overwritten)
    long long B;  // packed pairs n_in (n_in + 1) / 2
    int n_in, K, n_chan;
    int cpt;      // channels packed per 128-row tile (1, 2 or 4; n_in <= 128 / cpt)
};

// Tensor map of a planar FP16 operand [n_chan][npl][n_in][K] with boxes of
// (64 spectra x box_rows inputs), 128B swizzle (CUtensorMap storage, 128 bytes).
corr_status tma_encode_planar(void *tmap128, const void *planes, int n_in, int n_chan, int K, int npl,
                              int box_rows);
// One persistent launch over a precomputed work list (see batch.cu).
corr_status launch_xengine_tma_batch(const void *d_tmaps, const BatchSub *d_subs, const int4 *d_items,
                                     const int *d_cta_off, int grid, int *status, cudaStream_t st);

// F-engine split N = T1 x T2 (T1-point DFTs in pass 1 by T2 threads, T2-point DFTs in
// pass 2 by T1 threads); returns T2, or 0 for a length the F-engine does not support.
__host__ __device__ constexpr int fengine_t2(int n) {
    return n == 16 ? 4 : n == 64 ? 8 : n == 128 ? 16 : n == 256 ? 16 : n == 512 ? 32 : n == 1024 ? 32
         : n == 2048 ? 64 : n == 4096 ? 64 : 0;
}

// Bounded-wait iteration limit for device-side spins (mbarrier waits).
constexpr long long kSpinLimit = 1LL << 26;

}  // namespace corr
