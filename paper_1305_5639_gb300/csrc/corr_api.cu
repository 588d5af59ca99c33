// Host side of the libcorr C ABI: argument checking, handle state, buffer
// ownership and kernel dispatch. Every entry point returns a status code.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace corr {

static thread_local char g_last_error[512] = "";

void set_cuda_error(cudaError_t e, const char *what) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e),
                  cudaGetErrorString(e));
}

void set_error_text(const char *text) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", text); }

corr_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e, what);
        return CORR_ECUDA;
    }
    return CORR_OK;
}

StageScope::StageScope(const Handle &h, int stage, cudaStream_t st, int n_launch)
    : c_(h.clock), stage_(stage), st_(st) {
    if (!c_) return;
    c_->launches[stage] += n_launch;
    if (!c_->on) return;
    if (c_->recs.size() >= StageClock::kMaxRecs) {
        c_->overflow = true;
        return;
    }
    if (c_->pool.empty()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        c_->pool.push_back(e);
    }
    a_ = c_->pool.back();
    c_->pool.pop_back();
    if (cudaEventRecord(a_, st_) != cudaSuccess) {
        cudaGetLastError();
        c_->pool.push_back(a_);
        a_ = nullptr;
    }
}

StageScope::~StageScope() {
    if (!a_) return;
    cudaEvent_t b = nullptr;
    if (!c_->pool.empty()) {
        b = c_->pool.back();
        c_->pool.pop_back();
    } else if (cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        c_->pool.push_back(a_);
        return;
    }
    if (cudaEventRecord(b, st_) != cudaSuccess) {
        cudaGetLastError();
        c_->pool.push_back(a_);
        c_->pool.push_back(b);
        return;
    }
    c_->recs.push_back({stage_, a_, b});
}

namespace {

void free_clock(Handle &h) {
    if (!h.clock) return;
    for (cudaEvent_t e : h.clock->pool) cudaEventDestroy(e);
    for (const StageClock::Rec &r : h.clock->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete h.clock;
    h.clock = nullptr;
}

// NVTX range around a C-ABI call (visible in a profiler's timeline; a no-op when no
// tool is attached)
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

// Host-buffer pipeline resources (corr_fx_host): device copies, copy streams, events.
void free_fx(Handle &h) {
    cudaFree(h.fx_volt[0]);
    cudaFree(h.fx_volt[1]);
    cudaFree(h.fx_chan);
    h.fx_volt[0] = h.fx_volt[1] = h.fx_chan = nullptr;
    h.fx_par = 0;
    if (h.fx_in) cudaStreamDestroy(h.fx_in);
    if (h.fx_out) cudaStreamDestroy(h.fx_out);
    h.fx_in = h.fx_out = nullptr;
    for (cudaEvent_t &e : h.fx_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    h.fx_ready = false;
}

void free_buffers(Handle &h) {
    cudaFree(h.acc);
    cudaFree(h.vis64);
    cudaFree(h.twiddle);
    cudaFree(h.ftc_b);
    h.ftc_b = nullptr;
    cudaFree(h.dly_int);
    cudaFree(h.dly_ph);
    h.dly_int = nullptr;
    h.dly_ph = nullptr;
    cudaFree(h.pfb_win);
    cudaFree(h.pfb_y);
    h.pfb_win = nullptr;
    h.pfb_y = nullptr;
    cudaFree(h.status);
    cudaFree(h.power64);
    cudaFree(h.bwd_ws);
    cudaFree(h.planar_ws);
    h.planar_ws = nullptr;
    free_fx(h);
    if (h.bwd_side) cudaStreamDestroy(h.bwd_side);
    h.bwd_side = nullptr;
    for (cudaEvent_t &e : h.bwd_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    cudaFree(h.acc_alt);
    h.acc_alt = nullptr;
    h.dump_pending = false;
    h.pending_src = nullptr;
    h.acc = nullptr;
    h.vis64 = nullptr;
    h.twiddle = nullptr;
    h.status = nullptr;
    h.power64 = nullptr;
    h.bwd_ws = nullptr;
    free_clock(h);
}

bool use_tc(const Handle &h) {
    if (h.xengine == CORR_XENG_CUDACORE) return false;
    return h.precision != CORR_PREC_FP32;  // FP32 has no tensor-core X-engine
}

// Integration dumps are deferred into the next X-engine launch (whose idle warps run
// them; see corr_dump) where that launch is long enough to hide them: INT8 and FP16
// hi/lo on the tensor cores. Plain FP16's X-engine is too short for its FP32 dump
// (measured: a 2048-input step 37% slower deferred, hi/lo 7% faster, INT8 6% faster).
bool defer_ok(const Handle &h) {
    return (h.precision == CORR_PREC_INT8 || h.precision == CORR_PREC_FP16_HILO) && use_tc(h) &&
           !(h.flags & CORR_FLAG_FUSED_DUMP) && tma_available();
}

// Complete a deferred dump now (the dump kernel on the pending accumulator).
corr_status flush_dump(Handle &h, cudaStream_t st) {
    if (!h.dump_pending) return CORR_OK;
    const corr_status s = launch_dump_src(h, h.pending_src, st);
    if (s == CORR_OK) h.dump_pending = false;
    return s;
}

// Planar FP16 operands of the tensor-core X-engine: the caller's buffer itself
// (CORR_FLAG_PLANAR), or a conversion pass into the handle's workspace (complex
// int8 codes: exact; complex float: FP16 or the hi/lo split, with per-row scaling).
struct TcOperands {
    const void *planes = nullptr;
    int npl = 2;
    const float *row_scale = nullptr;
    int kstride = 0;
};

corr_status tc_operands(Handle &h, const void *chan_in, cudaStream_t st, TcOperands &op) {
    if (!tma_available()) {
        set_error_text("cuTensorMapEncodeTiled is not available from the driver");
        return CORR_EUNSUPPORTED;
    }
    if (h.flags & CORR_FLAG_PLANAR) {
        op.planes = chan_in;
        op.kstride = h.n_spectra;
        return CORR_OK;
    }
    op.npl = h.precision == CORR_PREC_FP16_HILO ? 4 : 2;
    const size_t need = planar_ws_bytes(h, op.npl);
    if (h.planar_ws_bytes < need) {
        cudaFree(h.planar_ws);
        h.planar_ws = nullptr;
        h.planar_ws_bytes = 0;
        if (cudaMalloc(&h.planar_ws, need) != cudaSuccess) {
            cudaGetLastError();
            set_error_text("allocating the planar FP16 operand workspace failed");
            return CORR_ENOMEM;
        }
        h.planar_ws_bytes = need;
    }
    op.planes = h.planar_ws;
    op.kstride = planar_kstride(h.n_spectra);
    StageScope sc(h, CORR_STAGE_PREP, st);
    if (h.precision == CORR_PREC_INT8) return launch_i8_to_planar(h, chan_in, h.planar_ws, st);
    op.row_scale = planar_row_scale(h, h.planar_ws, op.npl);
    return launch_to_planar(h, static_cast<const float2 *>(chan_in), h.planar_ws, op.npl, st);
}

}  // namespace
}  // namespace corr

using corr::Handle;

struct corr_s {
    Handle h;
};

namespace corr {

// corr_fx_host (out = the FP64 long integration) and corr_fx_host_accum (out = this
// integration's INT32 accumulator, copied while the dump adds it to the FP64 buffer:
// the dump only reads the accumulator).
static corr_status fx_host_run(corr_t *c, const void *volt_host, const float *chan_scale, void *out_host,
                               bool accum_out, void *stream) {
    if (!c || !volt_host || !chan_scale || !out_host) return CORR_EINVAL;
    Handle &h = c->h;
    if (h.precision != CORR_PREC_INT8 || !(h.flags & CORR_FLAG_PLANAR) || !corr::fengine_supported(h.n_chan))
        return CORR_EUNSUPPORTED;
    if (accum_out && (h.flags & CORR_FLAG_FUSED_DUMP)) return CORR_EUNSUPPORTED;  // no INT32 accumulator then
    corr::DeviceGuard dg(h.device);
    cudaStream_t st = corr::as_stream(stream);
    {
        const corr_status s = corr::flush_dump(h, st);  // this pipeline dumps per channel block itself
        if (s != CORR_OK) return s;
    }
    constexpr int NB = 8, NC = 8;  // input blocks (copy-in || F-engine), channel blocks (X + dump || copy-out)
    const size_t volt_bytes = (size_t)h.n_in * h.n_spectra * h.n_chan * 2;
    const size_t chan_bytes = (size_t)h.n_chan * 2 * h.n_in * h.n_spectra * 2;
    if (!h.fx_ready) {
        // all or nothing: a failed allocation or creation releases whatever this
        // attempt made, so that a retry starts again from scratch
        bool ok = cudaMalloc(&h.fx_volt[0], volt_bytes) == cudaSuccess &&
                  cudaMalloc(&h.fx_volt[1], volt_bytes) == cudaSuccess && cudaMalloc(&h.fx_chan, chan_bytes) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h.fx_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&h.fx_out, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t &e : h.fx_ev)
            ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            corr::free_fx(h);
            corr::set_error_text("corr_fx_host: allocating the device copies or creating the copy streams failed");
            return CORR_ENOMEM;
        }
        h.fx_ready = true;
    }
    // ev[1..NB]: input block b copied; ev[NB+1..NB+NC]: channel block dumped;
    // ev[NB+NC+1]: all copies out done; ev[NB+NC+2+p]: the F-engine has read device
    // copy p of the inputs (recorded by the call before the previous one, which used
    // the same copy). The copy-in waits only for that, not for `stream`, so that with
    // calls issued back to back it follows the previous call's copy-in directly,
    // overlapping that call's F-engine, X-engine and copy-out.
    cudaEvent_t *ev = h.fx_ev;
    const int par = h.fx_par;
    void *const vdev = h.fx_volt[par];
    CORR_CUDA_TRY(cudaStreamWaitEvent(h.fx_in, ev[NB + NC + 2 + par], 0));
    const size_t row = (size_t)h.n_spectra * h.n_chan * 2;  // bytes of one input's time series
    const int ib = (h.n_in + NB - 1) / NB;
    for (int b = 0; b < NB; ++b) {
        const int i0 = b * ib, i1 = std::min(h.n_in, i0 + ib);
        if (i1 > i0) {
            CORR_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(vdev) + row * i0,
                                          static_cast<const char *>(volt_host) + row * i0, row * (i1 - i0),
                                          cudaMemcpyHostToDevice, h.fx_in));
        }
        CORR_CUDA_TRY(cudaEventRecord(ev[1 + b], h.fx_in));
        CORR_CUDA_TRY(cudaStreamWaitEvent(st, ev[1 + b], 0));
        if (i1 <= i0) continue;  // fewer inputs than blocks: the last blocks are empty
        corr_status s = corr::launch_fengine_range(h, vdev, chan_scale, h.fx_chan, i0, i1 - i0, st);
        if (s != CORR_OK) return s;
    }
    CORR_CUDA_TRY(cudaEventRecord(ev[NB + NC + 2 + par], st));
    const bool fused = (h.flags & CORR_FLAG_FUSED_DUMP) != 0;
    const bool store = h.acc_zero;
    const int cb = (h.n_chan + NC - 1) / NC;
    for (int k = 0; k < NC; ++k) {
        const int c0 = k * cb, c1 = std::min(h.n_chan, c0 + cb);
        corr_status s = corr::launch_xengine_tma_range(h, h.fx_chan, 2, nullptr, nullptr, h.n_spectra, store, c0, c1,
                                                       st);
        if (s != CORR_OK) return s;
        const size_t off = (size_t)c0 * h.n_base;
        if (accum_out) {
            // copy the block's INT32 sums out while the dump adds them to the FP64 buffer
            CORR_CUDA_TRY(cudaEventRecord(ev[1 + NB + k], st));
            CORR_CUDA_TRY(cudaStreamWaitEvent(h.fx_out, ev[1 + NB + k], 0));
            if (c1 > c0)
                CORR_CUDA_TRY(cudaMemcpyAsync(static_cast<int2 *>(out_host) + off, static_cast<const int2 *>(h.acc) + off,
                                              sizeof(int2) * (size_t)(c1 - c0) * h.n_base, cudaMemcpyDeviceToHost,
                                              h.fx_out));
            if ((s = corr::launch_dump_range(h, c0, c1, st)) != CORR_OK) return s;
            continue;
        }
        if (!fused && (s = corr::launch_dump_range(h, c0, c1, st)) != CORR_OK) return s;
        CORR_CUDA_TRY(cudaEventRecord(ev[1 + NB + k], st));
        CORR_CUDA_TRY(cudaStreamWaitEvent(h.fx_out, ev[1 + NB + k], 0));
        if (c1 > c0)
            CORR_CUDA_TRY(cudaMemcpyAsync(static_cast<double2 *>(out_host) + off, h.vis64 + off,
                                          sizeof(double2) * (size_t)(c1 - c0) * h.n_base, cudaMemcpyDeviceToHost,
                                          h.fx_out));
    }
    CORR_CUDA_TRY(cudaEventRecord(ev[1 + NB + NC], h.fx_out));
    CORR_CUDA_TRY(cudaStreamWaitEvent(st, ev[1 + NB + NC], 0));
    h.acc_zero = true;
    h.acc_spectra = 0;
    h.fx_par = par ^ 1;
    return CORR_OK;
}

}  // namespace corr

extern "C" {

const char *corr_status_str(corr_status s) {
    switch (s) {
        case CORR_OK: return "CORR_OK";
        case CORR_EINVAL: return "CORR_EINVAL: invalid argument";
        case CORR_ENOMEM: return "CORR_ENOMEM: device allocation failed";
        case CORR_ECUDA: return "CORR_ECUDA: CUDA runtime error";
        case CORR_EOVERFLOW: return "CORR_EOVERFLOW: INT32 accumulator could overflow";
        case CORR_ESTATE: return "CORR_ESTATE: invalid call in the current state";
        case CORR_ETIMEOUT: return "CORR_ETIMEOUT: a device-side wait timed out";
        case CORR_EUNSUPPORTED: return "CORR_EUNSUPPORTED: unsupported shape or mode";
        default: return "CORR_?: unknown status";
    }
}

const char *corr_last_error(void) { return corr::g_last_error; }

int64_t corr_n_baselines(const corr_t *h) { return h ? h->h.n_base : -1; }

corr_status corr_create(int32_t n_ant, int32_t n_pol, int32_t n_chan, int32_t n_spectra, const corr_opts *opts,
                        corr_t **out) {
    if (!out) return CORR_EINVAL;
    *out = nullptr;
    if (n_ant <= 0 || n_pol <= 0 || n_chan <= 0 || n_spectra <= 0) return CORR_EINVAL;
    const int64_t n_in = (int64_t)n_ant * n_pol;
    if (n_in > 65535) {
        // the F-engine's grid holds one input per block row (at most 65535)
        corr::set_error_text("corr_create: n_ant * n_pol exceeds 65535 inputs");
        return CORR_EINVAL;
    }
    corr_opts o{CORR_PREC_FP32, CORR_XENG_AUTO, 0, -1};
    if (opts) o = *opts;
    if (o.precision < CORR_PREC_FP32 || o.precision > CORR_PREC_FP16_HILO) return CORR_EINVAL;
    if (o.xengine < CORR_XENG_AUTO || o.xengine > CORR_XENG_TCGEN05) return CORR_EINVAL;
    if ((o.flags & ~(CORR_FLAG_PLANAR | CORR_FLAG_FUSED_DUMP | CORR_FLAG_FENGINE_CUDACORE)) != 0) return CORR_EINVAL;
    // the dump fused into the X-engine epilogue exists on the tensor-core (TMA) X-engine:
    // INT8, FP16 and FP16 hi/lo on the AUTO or TCGEN05 X-engine
    if ((o.flags & CORR_FLAG_FUSED_DUMP) && (o.precision == CORR_PREC_FP32 || o.xengine == CORR_XENG_CUDACORE))
        return CORR_EUNSUPPORTED;
    if (o.precision == CORR_PREC_FP32 && o.xengine == CORR_XENG_TCGEN05) return CORR_EUNSUPPORTED;
    if ((o.flags & CORR_FLAG_PLANAR) &&
        (o.precision != CORR_PREC_INT8 || o.xengine == CORR_XENG_CUDACORE || (n_spectra % 8) != 0))
        return CORR_EUNSUPPORTED;
    if (o.precision == CORR_PREC_INT8) {
        // INT32 guard: |Re V| <= n_spectra * 2 * 128^2 (int8 codes include -128) must stay below 2^31
        if ((int64_t)n_spectra * 2 * 128 * 128 >= (int64_t)1 << 31) return CORR_EOVERFLOW;
    }
    if ((o.precision == CORR_PREC_FP16 || o.precision == CORR_PREC_FP16_HILO) && o.xengine == CORR_XENG_CUDACORE)
        return CORR_EUNSUPPORTED;

    corr_s *c = new (std::nothrow) corr_s();
    if (!c) return CORR_ENOMEM;
    Handle &h = c->h;
    h.n_ant = n_ant;
    h.n_pol = n_pol;
    h.n_in = (int32_t)n_in;
    h.n_chan = n_chan;
    h.n_spectra = n_spectra;
    h.n_base = n_in * (n_in + 1) / 2;
    h.precision = o.precision;
    h.xengine = o.xengine;
    h.flags = o.flags;
    if (o.device >= 0) {
        h.device = o.device;
    } else if (cudaGetDevice(&h.device) != cudaSuccess) {
        corr::set_cuda_error(cudaGetLastError(), "cudaGetDevice");
        delete c;
        return CORR_ECUDA;
    }
    corr::DeviceGuard dg(h.device);
    if (!dg.ok) {
        corr::set_cuda_error(cudaGetLastError(), "cudaSetDevice");
        delete c;
        return CORR_ECUDA;
    }
    if (cudaDeviceGetAttribute(&h.n_sm, cudaDevAttrMultiProcessorCount, h.device) != cudaSuccess) {
        corr::set_cuda_error(cudaGetLastError(), "cudaDeviceGetAttribute");
        delete c;
        return CORR_ECUDA;
    }
    const size_t nvis = (size_t)h.n_chan * (size_t)h.n_base;
    const size_t acc_bytes = nvis * 8;  // int2 or float2
    bool ok = cudaMalloc(&h.acc, acc_bytes) == cudaSuccess && cudaMalloc(&h.vis64, nvis * sizeof(double2)) == cudaSuccess &&
              cudaMalloc(&h.status, sizeof(int32_t)) == cudaSuccess &&
              cudaMalloc(&h.power64, sizeof(double) * (size_t)n_chan) == cudaSuccess;
    if (ok && corr::fengine_supported(n_chan)) ok = cudaMalloc(&h.twiddle, sizeof(float2) * (size_t)n_chan) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        corr::free_buffers(h);
        delete c;
        return CORR_ENOMEM;
    }
    ok = cudaMemset(h.acc, 0, acc_bytes) == cudaSuccess && cudaMemset(h.vis64, 0, nvis * sizeof(double2)) == cudaSuccess &&
         cudaMemset(h.status, 0, sizeof(int32_t)) == cudaSuccess;
    if (ok && h.twiddle) {
        // F-engine twiddles W_N^(t k1) = exp(-j 2 pi t k1 / N) for the N = T1 x T2 split,
        // laid out [k1][t] (k1 < T1, t < T2); computed in double, rounded once to float
        const int T2 = corr::fengine_t2(n_chan), T1 = n_chan / T2;
        std::vector<float2> tw((size_t)n_chan);
        for (int k1 = 0; k1 < T1; ++k1) {
            for (int t = 0; t < T2; ++t) {
                const int m = (t * k1) % n_chan;
                const double ang = 2.0 * M_PI * (double)m / (double)n_chan;
                tw[(size_t)k1 * T2 + t] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
            }
        }
        ok = cudaMemcpy(h.twiddle, tw.data(), sizeof(float2) * (size_t)n_chan, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (ok) {
        const corr_status s = corr::fengine_tc_init(h);
        if (s == CORR_ENOMEM) {
            corr::free_buffers(h);
            delete c;
            return CORR_ENOMEM;
        }
        ok = s == CORR_OK;
    }
    if (!ok) {
        corr::set_cuda_error(cudaGetLastError(), "corr_create init");
        corr::free_buffers(h);
        delete c;
        return CORR_ECUDA;
    }
    *out = c;
    return CORR_OK;
}

corr_status corr_set_delays(corr_t *c, const float *delays) {
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    if (!corr::fengine_supported(h.n_chan)) return CORR_EUNSUPPORTED;
    corr::DeviceGuard dg(h.device);
    // kernels already queued may still read the current tables
    CORR_CUDA_TRY(cudaDeviceSynchronize());
    if (!delays) {
        cudaFree(h.dly_int);
        cudaFree(h.dly_ph);
        h.dly_int = nullptr;
        h.dly_ph = nullptr;
        return CORR_OK;
    }
    const int N = h.n_chan;
    const int T2 = corr::fengine_t2(N), T1 = N / T2;
    std::vector<int32_t> D((size_t)h.n_in);
    std::vector<float2> ph((size_t)h.n_in * (T1 + T2));
    for (int i = 0; i < h.n_in; ++i) {
        const double t = (double)delays[i];
        if (!std::isfinite(t) || std::fabs(t) > 1.0e9) return CORR_EINVAL;
        // nearest integer, halves away from zero; the remainder f lies in [-0.5, 0.5]
        const double d = t >= 0 ? std::floor(t + 0.5) : -std::floor(-t + 0.5);
        const double f = t - d;
        D[(size_t)i] = (int32_t)d;
        // channel k = k1 + T1 k2: exp(+j 2 pi k f / N) = c[k1] d[k2]
        for (int k1 = 0; k1 < T1; ++k1) {
            const double a1 = 2.0 * M_PI * (double)k1 * f / (double)N;
            ph[(size_t)i * (T1 + T2) + k1] = make_float2((float)std::cos(a1), (float)std::sin(a1));
        }
        for (int k2 = 0; k2 < T2; ++k2) {
            const double a2 = 2.0 * M_PI * (double)T1 * (double)k2 * f / (double)N;
            ph[(size_t)i * (T1 + T2) + T1 + k2] = make_float2((float)std::cos(a2), (float)std::sin(a2));
        }
    }
    if (!h.dly_int) {
        if (cudaMalloc(&h.dly_int, sizeof(int32_t) * (size_t)h.n_in) != cudaSuccess ||
            cudaMalloc(&h.dly_ph, sizeof(float2) * ph.size()) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h.dly_int);
            h.dly_int = nullptr;
            h.dly_ph = nullptr;
            return CORR_ENOMEM;
        }
    }
    CORR_CUDA_TRY(cudaMemcpy(h.dly_int, D.data(), sizeof(int32_t) * D.size(), cudaMemcpyHostToDevice));
    CORR_CUDA_TRY(cudaMemcpy(h.dly_ph, ph.data(), sizeof(float2) * ph.size(), cudaMemcpyHostToDevice));
    return CORR_OK;
}

corr_status corr_set_pfb(corr_t *c, int32_t n_taps, const float *window) {
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    if (!corr::fengine_supported(h.n_chan)) return CORR_EUNSUPPORTED;
    corr::DeviceGuard dg(h.device);
    // kernels already queued may still read the current window
    CORR_CUDA_TRY(cudaDeviceSynchronize());
    if (!window) {
        cudaFree(h.pfb_win);
        cudaFree(h.pfb_y);
        h.pfb_win = nullptr;
        h.pfb_y = nullptr;
        h.pfb_taps = 0;
        return CORR_OK;
    }
    if (n_taps < 1 || n_taps > 64) return CORR_EINVAL;
    const size_t n = (size_t)n_taps * h.n_chan;
    for (size_t e = 0; e < n; ++e)
        if (!std::isfinite(window[e])) return CORR_EINVAL;
    cudaFree(h.pfb_win);
    h.pfb_win = nullptr;
    h.pfb_taps = 0;
    // the FIR output buffer: one complex FP32 frame per (input, spectrum)
    const size_t y_bytes = sizeof(float2) * (size_t)h.n_in * h.n_spectra * h.n_chan;
    if (!h.pfb_y && cudaMalloc(&h.pfb_y, y_bytes) != cudaSuccess) {
        cudaGetLastError();
        h.pfb_y = nullptr;
        return CORR_ENOMEM;
    }
    if (cudaMalloc(&h.pfb_win, sizeof(float) * n) != cudaSuccess) {
        cudaGetLastError();
        return CORR_ENOMEM;
    }
    CORR_CUDA_TRY(cudaMemcpy(h.pfb_win, window, sizeof(float) * n, cudaMemcpyHostToDevice));
    h.pfb_taps = n_taps;
    return CORR_OK;
}

corr_status corr_set_short_time(corr_t *c, int32_t block_spectra, int32_t *out) {
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    if (!out) {
        h.st_out = nullptr;
        h.st_block = 0;
        return CORR_OK;
    }
    if (h.precision != CORR_PREC_INT8 || !(h.flags & CORR_FLAG_PLANAR)) return CORR_EUNSUPPORTED;
    if (block_spectra < 64 || block_spectra > 512 || (block_spectra % 64) != 0 || (h.n_spectra % block_spectra) != 0)
        return CORR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(out) & 3u) != 0) return CORR_EINVAL;
    h.st_out = out;
    h.st_block = block_spectra;
    return CORR_OK;
}

corr_status corr_destroy(corr_t *c) {
    if (!c) return CORR_OK;
    corr::DeviceGuard dg(c->h.device);
    cudaDeviceSynchronize();
    corr::free_buffers(c->h);
    delete c;
    return CORR_OK;
}

corr_status corr_fengine(corr_t *c, const void *volt, const float *chan_scale, void *chan_out, void *stream) {
    corr::NvtxScope nvtx_("corr_fengine");
    if (!c || !volt || !chan_out) return CORR_EINVAL;
    Handle &h = c->h;
    if (!corr::fengine_supported(h.n_chan)) return CORR_EUNSUPPORTED;
    if (!corr::aligned16(volt) || !corr::aligned16(chan_out)) return CORR_EINVAL;
    if (h.precision == CORR_PREC_INT8) {
        if (!chan_scale) return CORR_EINVAL;
    } else if (chan_scale) {
        return CORR_EINVAL;
    }
    corr::DeviceGuard dg(h.device);
    return corr::launch_fengine(h, volt, chan_scale, chan_out, corr::as_stream(stream));
}

corr_status corr_fengine_power(corr_t *c, const void *volt, float *power, void *stream) {
    corr::NvtxScope nvtx_("corr_fengine_power");
    if (!c || !volt || !power) return CORR_EINVAL;
    Handle &h = c->h;
    if (!corr::fengine_supported(h.n_chan)) return CORR_EUNSUPPORTED;
    if (!corr::aligned16(volt)) return CORR_EINVAL;
    corr::DeviceGuard dg(h.device);
    return corr::launch_fengine_power(h, volt, power, corr::as_stream(stream));
}

corr_status corr_xengine(corr_t *c, const void *chan_in, const float *gains, void *stream) {
    corr::NvtxScope nvtx_("corr_xengine");
    if (!c || !chan_in) return CORR_EINVAL;
    Handle &h = c->h;
    if (!corr::aligned16(chan_in)) return CORR_EINVAL;
    if (gains && h.precision == CORR_PREC_INT8) return CORR_EINVAL;
    if (h.precision == CORR_PREC_INT8 && !(h.flags & CORR_FLAG_FUSED_DUMP)) {
        // the INT32 accumulator spans every call since the last dump
        if ((h.acc_spectra + h.n_spectra) * 2 * 128 * 128 >= (int64_t)1 << 31) return CORR_EOVERFLOW;
    }
    corr::DeviceGuard dg(h.device);
    const bool store = h.acc_zero;
    const float2 *g = reinterpret_cast<const float2 *>(gains);
    corr_status s;
    cudaStream_t st = corr::as_stream(stream);
    if (corr::use_tc(h)) {
        corr::TcOperands op;
        s = corr::tc_operands(h, chan_in, st, op);
        // a deferred dump of the previous integration rides along in this launch
        if (s == CORR_OK) s = corr::launch_xengine_tma(h, op.planes, op.npl, g, op.row_scale, op.kstride, store, st);
        if (s == CORR_OK) h.dump_pending = false;
    } else {
        s = corr::flush_dump(h, st);
        if (s == CORR_OK) s = corr::launch_xengine_cudacore(h, chan_in, g, store, st);
    }
    if (s == CORR_OK) {
        h.acc_zero = false;
        h.acc_spectra += h.n_spectra;
    }
    return s;
}

corr_status corr_xengine_cross(corr_t *c, const void *chan_in, const float *gains, int32_t p0, int32_t n_p,
                               int32_t q0, int32_t n_q, void *vis_out, void *stream) {
    corr::NvtxScope nvtx_("corr_xengine_cross");
    if (!c || !chan_in || !vis_out) return CORR_EINVAL;
    Handle &h = c->h;
    if (p0 < 0 || q0 < 0 || n_p <= 0 || n_q <= 0 || (int64_t)p0 + n_p > h.n_in || (int64_t)q0 + n_q > h.n_in)
        return CORR_EINVAL;
    if (!corr::aligned16(chan_in) || (reinterpret_cast<uintptr_t>(vis_out) & 7u) != 0) return CORR_EINVAL;
    if (gains && h.precision == CORR_PREC_INT8) return CORR_EINVAL;
    if (!corr::use_tc(h)) return CORR_EUNSUPPORTED;
    corr::DeviceGuard dg(h.device);
    cudaStream_t st = corr::as_stream(stream);
    corr::TcOperands op;
    corr_status s = corr::tc_operands(h, chan_in, st, op);
    if (s != CORR_OK) return s;
    return corr::launch_xengine_tma_rect(h, op.planes, op.npl, reinterpret_cast<const float2 *>(gains), op.row_scale,
                                         op.kstride, p0, n_p, q0, n_q, vis_out, st);
}

corr_status corr_get_accum(corr_t *c, void *out, void *stream) {
    corr::NvtxScope nvtx_("corr_get_accum");
    if (!c || !out) return CORR_EINVAL;
    Handle &h = c->h;
    if (h.flags & CORR_FLAG_FUSED_DUMP) return CORR_ESTATE;
    corr::DeviceGuard dg(h.device);
    const size_t bytes = (size_t)h.n_chan * h.n_base * 8;
    // after a dump (or reset) the accumulator is logically zero; its memory is only
    // overwritten by the next X-engine launch
    if (h.acc_zero) CORR_CUDA_TRY(cudaMemsetAsync(out, 0, bytes, corr::as_stream(stream)));
    else CORR_CUDA_TRY(cudaMemcpyAsync(out, h.acc, bytes, cudaMemcpyDeviceToDevice, corr::as_stream(stream)));
    return CORR_OK;
}

corr_status corr_dump(corr_t *c, double *vis_out, void *stream) {
    corr::NvtxScope nvtx_("corr_dump");
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    corr::DeviceGuard dg(h.device);
    cudaStream_t st = corr::as_stream(stream);
    if (!h.acc_zero && !(h.flags & CORR_FLAG_FUSED_DUMP)) {
        corr_status s = CORR_OK;
        bool deferred = false;
        if (!vis_out && !h.dump_pending && corr::defer_ok(h)) {
            // defer: the finished accumulator waits in pending_src and the next X-engine
            // launch, writing the other buffer, adds it to the FP64 buffer from idle warps
            if (!h.acc_alt && cudaMalloc(&h.acc_alt, (size_t)h.n_chan * h.n_base * 8) != cudaSuccess) {
                cudaGetLastError();
                h.acc_alt = nullptr;  // no second buffer: dump now
            }
            if (h.acc_alt) {
                h.pending_src = h.acc;
                std::swap(h.acc, h.acc_alt);
                h.dump_pending = true;
                deferred = true;
            }
        }
        if (!deferred) {
            s = corr::flush_dump(h, st);
            if (s == CORR_OK) s = corr::launch_dump(h, st);
        }
        if (s != CORR_OK) return s;
    }
    h.acc_zero = true;
    h.acc_spectra = 0;
    if (vis_out) {
        corr_status s = corr::flush_dump(h, st);
        if (s != CORR_OK) return s;
        CORR_CUDA_TRY(cudaMemcpyAsync(vis_out, h.vis64, (size_t)h.n_chan * h.n_base * sizeof(double2),
                                      cudaMemcpyDeviceToDevice, st));
    }
    return CORR_OK;
}

corr_status corr_restore_vis(corr_t *c, const double *vis_in, void *stream) {
    corr::NvtxScope nvtx_("corr_restore_vis");
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    if (vis_in && !corr::aligned16(vis_in)) return CORR_EINVAL;
    corr::DeviceGuard dg(h.device);
    cudaStream_t st = corr::as_stream(stream);
    const size_t bytes = (size_t)h.n_chan * h.n_base * sizeof(double2);
    if (vis_in) CORR_CUDA_TRY(cudaMemcpyAsync(h.vis64, vis_in, bytes, cudaMemcpyDeviceToDevice, st));
    else CORR_CUDA_TRY(cudaMemsetAsync(h.vis64, 0, bytes, st));
    h.dump_pending = false;  // the buffer it would have added to is replaced
    h.acc_zero = true;
    h.acc_spectra = 0;
    return CORR_OK;
}

corr_status corr_flush(corr_t *c, void *stream) {
    corr::NvtxScope nvtx_("corr_flush");
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    corr::DeviceGuard dg(h.device);
    return corr::flush_dump(h, corr::as_stream(stream));
}

corr_status corr_selftest_bounded_wait(int32_t device, int64_t limit_ns) {
    if (limit_ns < 1000000 || limit_ns > 1000000000) return CORR_EINVAL;
    int n_dev = 0;
    CORR_CUDA_TRY(cudaGetDeviceCount(&n_dev));
    if (device < 0 || device >= n_dev) return CORR_EINVAL;
    corr::DeviceGuard dg(device);
    return corr::selftest_bounded_wait((uint64_t)limit_ns);
}

corr_status corr_fx_host(corr_t *c, const void *volt_host, const float *chan_scale, double *vis_host, void *stream) {
    corr::NvtxScope nvtx_("corr_fx_host");
    return corr::fx_host_run(c, volt_host, chan_scale, vis_host, false, stream);
}

corr_status corr_fx_host_accum(corr_t *c, const void *volt_host, const float *chan_scale, int32_t *acc_host,
                               void *stream) {
    corr::NvtxScope nvtx_("corr_fx_host_accum");
    return corr::fx_host_run(c, volt_host, chan_scale, acc_host, true, stream);
}

corr_status corr_check_status(corr_t *c, void *stream) {
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    corr::DeviceGuard dg(h.device);
    int32_t v = 0;
    cudaStream_t st = corr::as_stream(stream);
    CORR_CUDA_TRY(cudaMemcpyAsync(&v, h.status, sizeof(v), cudaMemcpyDeviceToHost, st));
    CORR_CUDA_TRY(cudaStreamSynchronize(st));
    if (v != 0) {
        CORR_CUDA_TRY(cudaMemsetAsync(h.status, 0, sizeof(int32_t), st));
        return (corr_status)v;
    }
    return CORR_OK;
}

corr_status corr_set_stage_timing(corr_t *c, int32_t on) {
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    if (!h.clock) {
        h.clock = new (std::nothrow) corr::StageClock();
        if (!h.clock) return CORR_ENOMEM;
    }
    h.clock->on = on != 0;
    return CORR_OK;
}

corr_status corr_stage_times(corr_t *c, double *ms, int64_t *launches) {
    if (!c || !ms) return CORR_EINVAL;
    Handle &h = c->h;
    for (int k = 0; k < CORR_STAGE_COUNT; ++k) {
        ms[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    if (!h.clock) return CORR_OK;
    corr::DeviceGuard dg(h.device);
    corr::StageClock &ck = *h.clock;
    corr_status result = CORR_OK;
    for (const corr::StageClock::Rec &r : ck.recs) {
        float t = 0.f;
        if (result == CORR_OK) {
            cudaError_t e = cudaEventSynchronize(r.b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
            if (e != cudaSuccess) {
                corr::set_cuda_error(e, "corr_stage_times");
                result = CORR_ECUDA;
            }
        }
        ms[r.stage] += (double)t;
        ck.pool.push_back(r.a);
        ck.pool.push_back(r.b);
    }
    ck.recs.clear();
    if (launches)
        for (int k = 0; k < CORR_STAGE_COUNT; ++k) launches[k] = ck.launches[k];
    for (int64_t &n : ck.launches) n = 0;
    if (result == CORR_OK && ck.overflow) {
        corr::set_error_text("corr_stage_times: more than 65536 stage records since the last read");
        result = CORR_ESTATE;
    }
    ck.overflow = false;
    return result;
}

corr_status corr_reset(corr_t *c, void *stream) {
    if (!c) return CORR_EINVAL;
    Handle &h = c->h;
    corr::DeviceGuard dg(h.device);
    cudaStream_t st = corr::as_stream(stream);
    const size_t nvis = (size_t)h.n_chan * h.n_base;
    CORR_CUDA_TRY(cudaMemsetAsync(h.acc, 0, nvis * 8, st));
    CORR_CUDA_TRY(cudaMemsetAsync(h.vis64, 0, nvis * sizeof(double2), st));
    h.dump_pending = false;
    h.acc_zero = true;
    h.acc_spectra = 0;
    return CORR_OK;
}

corr_status corr_backward(corr_t *c, const float *grad_vis, const void *chan_in, const float *gains, float *grad_chan,
                          float *grad_gains, void *stream) {
    corr::NvtxScope nvtx_("corr_backward");
    if (!c || !grad_vis || !chan_in) return CORR_EINVAL;
    Handle &h = c->h;
    if (h.precision != CORR_PREC_FP32 && h.precision != CORR_PREC_FP16_HILO) return CORR_ESTATE;
    if (!grad_chan && !grad_gains) return CORR_OK;
    if (!corr::aligned16(chan_in) || (grad_chan && !corr::aligned16(grad_chan))) return CORR_EINVAL;
    corr::DeviceGuard dg(h.device);
    if (h.precision == CORR_PREC_FP16_HILO) {
        // tensor cores, FP16 hi/lo split (dX GEMM on tcgen05)
        if (!corr::xengine_tma_supported(h) || (h.n_in % 8) != 0) return CORR_EUNSUPPORTED;
        const size_t need = corr::backward_tc_workspace_bytes(h, nullptr);
        if (h.bwd_ws_bytes < need) {
            cudaFree(h.bwd_ws);
            h.bwd_ws = nullptr;
            h.bwd_ws_bytes = 0;
            if (cudaMalloc(&h.bwd_ws, need) != cudaSuccess) {
                cudaGetLastError();
                return CORR_ENOMEM;
            }
            h.bwd_ws_bytes = need;
        }
        if (!h.bwd_side) {
            cudaStream_t side = nullptr;
            bool ok = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) == cudaSuccess;
            for (cudaEvent_t &e : h.bwd_ev)
                ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
            if (!ok) {
                // all or nothing, so that a retry creates everything again
                cudaGetLastError();
                if (side) cudaStreamDestroy(side);
                for (cudaEvent_t &e : h.bwd_ev) {
                    if (e) cudaEventDestroy(e);
                    e = nullptr;
                }
                corr::set_error_text("corr_backward: creating the side stream or its events failed");
                return CORR_ECUDA;
            }
            h.bwd_side = side;
        }
        return corr::launch_backward_tc(h, reinterpret_cast<const float2 *>(grad_vis),
                                        static_cast<const float2 *>(chan_in), reinterpret_cast<const float2 *>(gains),
                                        reinterpret_cast<float2 *>(grad_chan), reinterpret_cast<float2 *>(grad_gains),
                                        h.bwd_ws, corr::as_stream(stream), h.bwd_side, h.bwd_ev);
    }
    if (grad_gains) {
        const size_t need = corr::backward_workspace_bytes(h);
        if (h.bwd_ws_bytes < need) {
            cudaFree(h.bwd_ws);
            h.bwd_ws = nullptr;
            h.bwd_ws_bytes = 0;
            if (cudaMalloc(&h.bwd_ws, need) != cudaSuccess) {
                cudaGetLastError();
                return CORR_ENOMEM;
            }
            h.bwd_ws_bytes = need;
        }
    }
    return corr::launch_backward_ws(h, reinterpret_cast<const float2 *>(grad_vis),
                                    static_cast<const float2 *>(chan_in), reinterpret_cast<const float2 *>(gains),
                                    reinterpret_cast<float2 *>(grad_chan), reinterpret_cast<float2 *>(grad_gains),
                                    h.bwd_ws, corr::as_stream(stream));
}

}  // extern "C"
