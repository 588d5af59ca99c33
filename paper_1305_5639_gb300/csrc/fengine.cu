// F-engine host entry points: launch selection by front-end feature, the per-channel
// power pass and the allocation-free power pass. The kernel is in fengine_kernel.cuh.
#include <cmath>
#include <cstdio>
#include <initializer_list>

#include "fengine_kernel.cuh"

namespace corr {
namespace {

template <int MODE>
corr_status dispatch(const FShape &f, const void *volt, const float *scale, void *out, double *power,
                     cudaStream_t st) {
    if (f.dint || f.dph) return fengine_run_delay(MODE, f, volt, scale, out, power, st);
    return fengine_run_plain(MODE, f, volt, scale, out, power, st);
}

FShape shape_of(const Handle &h) {
    FShape f{h.n_in, h.n_chan, h.n_spectra, h.precision == CORR_PREC_INT8, h.twiddle};
    if (h.dly_int) {
        f.dint = h.dly_int;
        f.dph = h.dly_ph;
    }
    return f;
}

// With the polyphase filter bank the FIR pass forms the tap-weighted frames of inputs
// [f.i0, f.i0 + n_run) (applying the integer delay advance) into the handle's complex
// FP32 buffer, and the FFT pass then reads those (float input, phase only).
corr_status pfb_front(const Handle &h, FShape &f, const void *&volt, cudaStream_t st) {
    if (!h.pfb_win) return CORR_OK;
    StageScope sc(h, CORR_STAGE_PFB, st);
    const corr_status s = launch_pfb_fir(h, volt, f.i0, f.n_run < 0 ? f.n_in : f.n_run, st);
    if (s != CORR_OK) return s;
    volt = h.pfb_y;
    f.i8 = false;
    f.dint = nullptr;
    return CORR_OK;
}

__global__ void k_power_finalize(const double *__restrict__ p64, float *__restrict__ out, int n, double inv) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = (float)(p64[k] * inv);
}

// Per-channel power: zero the FP64 accumulators, run the FFT pass, scale to a mean.
corr_status power_pass(const FShape &f, const void *volt, double *acc64, float *power, cudaStream_t st) {
    CORR_CUDA_TRY(cudaMemsetAsync(acc64, 0, sizeof(double) * f.n_chan, st));
    corr_status s = dispatch<kPower>(f, volt, nullptr, nullptr, acc64, st);
    if (s != CORR_OK) return s;
    const double inv = 1.0 / (2.0 * (double)f.n_in * (double)f.n_spectra);
    k_power_finalize<<<(f.n_chan + 255) / 256, 256, 0, st>>>(acc64, power, f.n_chan, inv);
    return check_launch("k_power_finalize");
}

}  // namespace

bool fengine_supported(int n) { return fengine_t2(n) > 0; }

corr_status launch_fengine_range(const Handle &h, const void *volt, const float *scale, void *out, int i0, int n_run,
                                 cudaStream_t st) {
    // inputs [i0, i0 + n_run), or all of them for n_run < 0 (then i0 = 0)
    if (n_run < 0 ? i0 != 0 : (i0 < 0 || (long long)i0 + n_run > h.n_in)) {
        set_error_text("F-engine input range outside the handle's inputs");
        return CORR_EINVAL;
    }
    FShape f = shape_of(h);
    f.i0 = i0;
    f.n_run = n_run;
    if (n_run == 0) return CORR_OK;
    corr_status s = pfb_front(h, f, volt, st);
    if (s != CORR_OK) return s;
    StageScope sc(h, CORR_STAGE_FENGINE, st);
    if (fengine_tc_applies(h)) return launch_fengine_tc(h, volt, scale, out, i0, n_run, st);
    if (h.precision == CORR_PREC_INT8 && (h.flags & CORR_FLAG_PLANAR))
        return dispatch<kRequantPlanar>(f, volt, scale, out, nullptr, st);
    if (h.precision == CORR_PREC_INT8) return dispatch<kRequant>(f, volt, scale, out, nullptr, st);
    return dispatch<kFloatOut>(f, volt, nullptr, out, nullptr, st);
}

corr_status launch_fengine(const Handle &h, const void *volt, const float *scale, void *out,
                           cudaStream_t st) {
    return launch_fengine_range(h, volt, scale, out, 0, -1, st);
}

corr_status launch_fengine_power(const Handle &h, const void *volt, float *power, cudaStream_t st) {
    FShape f = shape_of(h);
    corr_status s = pfb_front(h, f, volt, st);
    if (s != CORR_OK) return s;
    StageScope sc(h, CORR_STAGE_POWER, st, 2);
    return power_pass(f, volt, h.power64, power, st);
}

// ------------------------------------------------------------------ allocation-free power pass
//
// corr_fengine_power_noalloc runs the same per-channel power pass as
// corr_fengine_power without a handle and without allocating device memory. Its
// scratch (the FP64 per-channel accumulators) and its twiddle tables live in
// file-scope __device__ arrays that every GPU loading this library holds until
// the process exits. The twiddle tables are constant-initialised (computed at
// compile time), so they are in place whenever the module is loaded, in any
// context. Host code only sees a host-side stand-in for those arrays, so each
// call looks their device addresses up with cudaGetSymbolAddress (which allocates
// nothing) and passes them to the kernels.
namespace {

constexpr int kNaMaxChan = 1024;  // largest n_chan the static scratch holds (8 KB of FP64)
constexpr int kNaTwTotal = 16 + 64 + 256 + 1024;

constexpr int na_tw_offset(int n) {
    return n == 16 ? 0 : n == 64 ? 16 : n == 256 ? 80 : n == 1024 ? 336 : -1;
}

// F-engine twiddle tables W_N^(t k1) = exp(-j 2 pi t k1 / N), [k1][t] layout with
// N = T x T, for N = 16, 64, 256 and 1024, as (re, im) float pairs.
struct NaTwiddles {
    float v[2 * kNaTwTotal];
};

constexpr NaTwiddles na_make_twiddles() {
    NaTwiddles r{};
    for (int n : {16, 64, 256, 1024}) {
        int T = 1;
        while (T * T < n) T *= 2;
        const int o = na_tw_offset(n);
        for (int k1 = 0; k1 < T; ++k1)
            for (int t = 0; t < T; ++t) {
                const int j = (t * k1) % n;
                r.v[2 * (o + k1 * T + t)] = (float)cos2pi(j, n);
                r.v[2 * (o + k1 * T + t) + 1] = (float)-sin2pi(j, n);
            }
    }
    return r;
}

// FP64 power accumulators, shared by every call on a device (cleared per call).
static __device__ __align__(256) double g_na_power[kNaMaxChan];
static __device__ __align__(256) NaTwiddles g_na_tw = na_make_twiddles();

corr_status na_reject(const char *why) {
    set_error_text(why);
    return CORR_EINVAL;
}

}  // namespace
}  // namespace corr

extern "C" corr_status corr_fengine_power_noalloc(const void *volt, int32_t n_in, int32_t n_chan,
                                                   int32_t n_spectra, int32_t precision, float *power,
                                                   void *stream) {
    using corr::na_reject;
    if (!volt || !power) return na_reject("corr_fengine_power_noalloc: null volt or power");
    if (n_in <= 0 || n_chan <= 0 || n_spectra <= 0)
        return na_reject("corr_fengine_power_noalloc: n_in, n_chan and n_spectra must be positive");
    if (n_in > 65535) return na_reject("corr_fengine_power_noalloc: n_in exceeds 65535 inputs");
    if (n_chan > corr::kNaMaxChan)
        return na_reject("corr_fengine_power_noalloc: n_chan exceeds the 1024-channel static scratch");
    if (corr::na_tw_offset(n_chan) < 0) {
        corr::set_error_text("corr_fengine_power_noalloc: n_chan must be 16, 64, 256 or 1024");
        return CORR_EUNSUPPORTED;
    }
    if (precision != CORR_PREC_INT8 && precision != CORR_PREC_FP32)
        return na_reject("corr_fengine_power_noalloc: precision must be CORR_PREC_INT8 or CORR_PREC_FP32");
    if ((reinterpret_cast<uintptr_t>(volt) & 15u) != 0)
        return na_reject("corr_fengine_power_noalloc: volt must be 16-byte aligned");
    // device addresses of the static arrays in the current context (no allocation)
    double *pw = nullptr;
    corr::NaTwiddles *tw = nullptr;
    CORR_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&pw), corr::g_na_power));
    CORR_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void **>(&tw), corr::g_na_tw));
    const corr::FShape f{n_in, n_chan, n_spectra, precision == CORR_PREC_INT8,
                         reinterpret_cast<const float2 *>(tw) + corr::na_tw_offset(n_chan)};  // v at offset 0
    return corr::power_pass(f, volt, pw, power, static_cast<cudaStream_t>(stream));
}
