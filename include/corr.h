/*
 * corr.h -- C ABI of libcorr, a single-GPU (sm_103a) FX correlator.
 *
 * The library computes the data-parallel hot path of the FX correlator described
 * in Wang & Harris (2013), Section 2:
 *   F-engine (Eq. 1): per input, per spectrum a, S_a,i[k] = sum_{n<N} s_i[aN+n] e^{-j 2 pi k n / N},
 *                     unnormalised, bins 0..N-1 in natural order, no window;
 *   X-engine (Eq. 2): per channel k, V_ij[k] = sum_a S_a,i[k] conj(S_a,j[k]) for all
 *                     i >= j (autocorrelations included: the "triangle" of Section 4).
 * The library emits V_ij = conj(C_ij) of Eq. 2 (the conjugate sits on the second
 * index); magnitudes and autocorrelations are identical.
 *
 * Conventions for every entry point:
 *   - n_in = n_ant * n_pol inputs; input index i = ant * n_pol + pol.
 *   - B = n_in (n_in + 1) / 2 packed visibilities per channel, packed index
 *     b(i, j) = i (i + 1) / 2 + j for i >= j.
 *   - Complex values are interleaved (re, im): complex int8 = 2 x int8,
 *     complex float = float2, complex double = double2.
 *   - All data pointers are DEVICE pointers owned by the caller unless stated; the
 *     library owns the integration accumulator, the FP64 long-integration buffer,
 *     twiddle tables and status words, and frees them in corr_destroy.
 *   - All calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) and return a status code; they never abort the process.
 *     Argument errors are reported before anything is enqueued.
 *   - A handle is not thread-safe: calls on one handle must be serialised by the
 *     caller (they may use different streams if the caller orders them).
 */
#ifndef CORR_H
#define CORR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CORR_API __attribute__((visibility("default")))
#else
#define CORR_API
#endif

typedef struct corr_s corr_t;
typedef int32_t corr_status;

enum {
    CORR_OK = 0,
    CORR_EINVAL = 1,       /* bad argument (null, size, alignment, precision mismatch) */
    CORR_ENOMEM = 2,       /* device allocation failed */
    CORR_ECUDA = 3,        /* a CUDA runtime call failed; see corr_last_error() */
    CORR_EOVERFLOW = 4,    /* INT32 integration accumulator could overflow */
    CORR_ESTATE = 5,       /* call not valid in the handle's current state */
    CORR_ETIMEOUT = 6,     /* a bounded device-side wait gave up (kernel returned early) */
    CORR_EUNSUPPORTED = 7  /* shape or mode not supported by this build */
};

/* Arithmetic of the X-engine. The FP16 forms first scale each (channel, input)
 * row of the input by a power of two 2^e that brings its largest component into
 * [2^14, 2^15) (exact, undone on the output), so that their accuracy does not
 * depend on the data's magnitude. */
enum {
    CORR_PREC_FP32 = 0,      /* float input, FP32 CUDA-core FFMA */
    CORR_PREC_INT8 = 1,      /* complex int8 input, exact integer result (INT32) */
    CORR_PREC_FP16 = 2,      /* float input rounded to FP16, FP32 accumulation (tensor cores) */
    CORR_PREC_FP16_HILO = 3  /* float input split x 2^e = h + l into two FP16 parts, h = fp16(x 2^e),
                                l = fp16(x 2^e - h); V ~ hh + hl + lh, FP32 accumulation (tensor cores) */
};

/* X-engine implementation. AUTO picks tcgen05 tensor cores for INT8/FP16/FP16_HILO
 * and CUDA cores for FP32 (TCGEN05 with FP32 is CORR_EUNSUPPORTED). The tensor-core
 * X-engine reads planar FP16 operands by TMA: the caller's own (CORR_FLAG_PLANAR)
 * or ones the library converts the input into, in a workspace allocated on first
 * use (4 bytes per complex sample, 8 for FP16_HILO). CUDACORE with INT8 uses exact
 * dp4a integer arithmetic. */
enum { CORR_XENG_AUTO = 0, CORR_XENG_CUDACORE = 1, CORR_XENG_TCGEN05 = 2 };

/* Layout flags (corr_opts.flags).
 * CORR_FLAG_PLANAR (INT8 only): channelised data is exchanged in the planar FP16
 *   layout [n_chan][2][n_in][n_spectra] (plane 0 = Re, plane 1 = Im; 2 bytes per
 *   component) instead of complex int8. The values are the same int8 codes, held
 *   exactly in FP16, so results are unchanged; the X-engine then streams its
 *   operands straight into shared memory with TMA. Requires n_spectra % 8 == 0
 *   (CORR_EUNSUPPORTED otherwise); doubles the channelised buffer's size. */
enum { CORR_FLAG_PLANAR = 1 };

/* CORR_FLAG_FUSED_DUMP: corr_xengine adds each integration straight into the FP64
 *   long-integration buffer from its epilogue. Valid on the tensor-core X-engine
 *   (INT8, FP16, FP16_HILO with xengine AUTO or TCGEN05): for INT8 the sums are
 *   exact, so the FP64 sums equal a separate dump's; for FP16 the same FP32 tile
 *   sums a separate dump would add. CORR_EUNSUPPORTED otherwise (FP32, CUDACORE).
 *   There is then no integration accumulator: corr_get_accum returns CORR_ESTATE,
 *   and corr_dump only copies the FP64 buffer out. */
enum { CORR_FLAG_FUSED_DUMP = 2 };

/* CORR_FLAG_FENGINE_CUDACORE: run the F-engine's FFT on the CUDA cores even where the
 *   tensor-core F-engine applies. By default, INT8 handles with n_chan = 1024 and
 *   neither delay compensation nor the filter bank channelise with tcgen05: the two
 *   32-point DFT stages of the 32 x 32 split of Eq. 1 as FP16 hi/lo GEMMs with FP32
 *   accumulation (the twiddles and the hi/lo split of the intermediate in FP32). Both
 *   forms round each code from an FP32-accurate spectrum; a code may differ by one
 *   between them only where the scaled value lies within that error of a rounding
 *   boundary. */
enum { CORR_FLAG_FENGINE_CUDACORE = 4 };

typedef struct corr_opts {
    int32_t precision; /* CORR_PREC_*, default CORR_PREC_FP32 */
    int32_t xengine;   /* CORR_XENG_*, default CORR_XENG_AUTO */
    int32_t flags;     /* CORR_FLAG_* bits, default 0 */
    int32_t device;    /* CUDA device ordinal; -1 = the current device */
} corr_opts;

/* Create a correlator for n_ant x n_pol inputs, an n_chan-point FFT (n_chan
 * channels) and n_spectra spectra per integration (Section 2: the streams, the
 * FFT length and the A spectra of one accumulation; the handle itself, its
 * precisions and flags have no counterpart in the paper). opts may be NULL
 * (FP32, AUTO, current device). n_ant * n_pol <= 65535 (CORR_EINVAL otherwise).
 * The F-engine supports n_chan in {16, 64, 128, 256, 512, 1024, 2048, 4096}; the
 * X-engine any n_chan >= 1. For INT8, n_spectra * 2 * 128^2 must stay below 2^31
 * (int8 codes include -128; CORR_EOVERFLOW otherwise). *out receives the handle
 * (NULL on error). */
CORR_API corr_status corr_create(int32_t n_ant, int32_t n_pol, int32_t n_chan, int32_t n_spectra,
                        const corr_opts *opts, corr_t **out);

/* Free every library-owned buffer (no counterpart in the paper). Synchronises the
 * device. NULL is accepted. */
CORR_API corr_status corr_destroy(corr_t *h);

/* Static string for a status code. */
CORR_API const char *corr_status_str(corr_status s);

/* Text of the last CUDA error seen on this thread ("" if none). */
CORR_API const char *corr_last_error(void);

/* Number of packed visibilities per channel, n_in (n_in + 1) / 2. */
CORR_API int64_t corr_n_baselines(const corr_t *h);

/* F-engine, Eq. 1 (Section 2), for one integration.
 *   volt      [n_in][n_spectra * n_chan] complex time series; spectrum a of input i
 *             is samples a*n_chan .. a*n_chan + n_chan - 1. Complex int8 for
 *             CORR_PREC_INT8 (the paper's 8-bit streams, Section 5), complex float
 *             otherwise. 16-byte aligned.
 *   chan_scale [n_chan] float, INT8 only (must be NULL otherwise): per-channel
 *             re-quantisation scale. Each of Re, Im of S * scale_k is clamped to
 *             [-127, 127] and rounded half-to-even to int8 (8-bit packing of the
 *             expanded spectra, Section 6.2).
 *   chan_out  [n_chan][n_in][n_spectra] channel-major ("corner-turned") output:
 *             complex int8 for INT8, complex float (FP32 FFT, unnormalised)
 *             otherwise; with CORR_FLAG_PLANAR the planar FP16 layout
 *             [n_chan][2][n_in][n_spectra]. 16-byte aligned. */
CORR_API corr_status corr_fengine(corr_t *h, const void *volt, const float *chan_scale, void *chan_out,
                         void *stream);

/* Delay compensation fused into the F-engine (a station-based function the paper
 * leaves for future work, Section 7). delays: host [n_in] float, the delay tau_i
 * of input i in samples (|tau_i| <= 1e9), or NULL to switch compensation off.
 * With D_i the nearest integer to tau_i (halves away from zero) and f_i = tau_i - D_i,
 * corr_fengine and corr_fengine_power then channelise the advanced stream
 * s'_i[t] = s_i[t + D_i] (zero where t + D_i lies outside the n_spectra * n_chan
 * recorded samples) and multiply channel k (natural order 0..n_chan-1) by
 * exp(+j 2 pi k f_i / n_chan); a tone at a bin frequency delayed by tau_i then has
 * zero phase. The tables live on the device with the handle. Synchronises the
 * device (kernels already queued may use the previous tables). Returns
 * CORR_EUNSUPPORTED when n_chan has no F-engine, CORR_EINVAL for a non-finite or
 * out-of-range delay. */
CORR_API corr_status corr_set_delays(corr_t *h, const float *delays);

/* Polyphase filter-bank front end for the F-engine (a windowed multi-tap
 * channeliser; the paper's F-engine is a plain FFT, Section 5). window: host
 * [n_taps][n_chan] float weights h[p][n] (1 <= n_taps <= 64), or NULL to switch the
 * filter bank off. corr_fengine and corr_fengine_power then transform, for spectrum
 * a of input i, the frame y[n] = sum_p h[p][n] s'_i[(a + p) n_chan + n] (s'_i the
 * stream after any delay compensation, zero past the record, so each input keeps
 * n_spectra spectra; with delays the per-channel phase follows the transform).
 * Synchronises the device. CORR_EUNSUPPORTED when n_chan has no F-engine,
 * CORR_EINVAL for a bad tap count or a non-finite weight. */
CORR_API corr_status corr_set_pfb(corr_t *h, int32_t n_taps, const float *window);

/* Per-channel mean power per real component of the F-engine spectra,
 * power[k] = sum_{i,a} |S_a,i[k]|^2 / (2 n_in n_spectra), in FP32 (atomics; not
 * bit-reproducible). Used to set chan_scale = target_rms / sqrt(power).
 *   volt as for corr_fengine; power [n_chan] float (device), overwritten. */
CORR_API corr_status corr_fengine_power(corr_t *h, const void *volt, float *power, void *stream);

/* The per-channel power pass of corr_fengine_power for callers that cannot
 * allocate device memory: it takes no handle and calls no cudaMalloc, cudaFree
 * or other allocating routine. (The paper has no counterpart; this serves hosts
 * that own all device memory themselves, e.g. a real-time pipeline whose memory
 * is fixed up front, or code where an allocation's implicit synchronisation
 * would stall other streams.)
 *   volt      [n_in][n_spectra * n_chan] raw voltages, complex int8 when
 *             precision == CORR_PREC_INT8, complex float when CORR_PREC_FP32;
 *             16-byte aligned, device.
 *   power     [n_chan] float, device: sum_{i,a} |S_a,i[k]|^2 / (2 n_in n_spectra).
 * n_chan must be one of 16, 64, 256, 1024: larger values are rejected with
 * CORR_EINVAL (the static scratch holds 1024 FP64 accumulators), others with
 * CORR_EUNSUPPORTED; n_in must be at most 65535 (CORR_EINVAL). Every rejection
 * sets corr_last_error(). The scratch and the (compile-time) twiddle tables are
 * file-scope device arrays (about 19 KB) that each GPU loading the library keeps
 * until the process exits. Each call looks up their device addresses in the
 * current context (no allocation); the first call on a device may load the
 * library's device code, so make it before any stream capture. All calls on a
 * device share the scratch and clear it first: calls that overlap on the GPU race,
 * so serialise them (one stream, or events). Runs on the current device and
 * `stream`. */
CORR_API corr_status corr_fengine_power_noalloc(const void *volt, int32_t n_in, int32_t n_chan,
                                                int32_t n_spectra, int32_t precision, float *power,
                                                void *stream);

/* X-engine, Eq. 2 (Section 2), for one integration of n_spectra spectra: adds
 * V'_ij[k] = g_i conj(g_j) sum_a X_a,i[k] conj(X_a,j[k]) (i >= j) into the
 * library-owned integration accumulator.
 *   chan_in [n_chan][n_in][n_spectra]: complex int8 for INT8, complex float
 *           otherwise (the FP16 paths scale, round or split it in a conversion
 *           pass); with CORR_FLAG_PLANAR the planar FP16 layout. 16-byte aligned.
 *   gains   [n_in] complex float, or NULL for unit gains. Not allowed with INT8
 *           (the INT8 result is an exact integer; CORR_EINVAL).
 * INT8: accumulator is INT32 per component; CORR_EOVERFLOW if the spectra
 * accumulated since the last dump would exceed the INT32 guard. */
CORR_API corr_status corr_xengine(corr_t *h, const void *chan_in, const float *gains, void *stream);

/* Short-time visibilities for a transient detector (a hook between the
 * cross-multiplication and the accumulation; the paper lists transient detection
 * as future work, Section 7). With out set, every corr_xengine call (and the
 * X-engine of corr_fx_host) also writes the visibilities of each block of
 * block_spectra consecutive spectra, before they are summed into the integration:
 *   out [n_spectra / block_spectra][n_chan][2][B] int32: per block and channel the
 *       Re plane then the Im plane of the packed lower triangle; exact integers,
 *       whose sum over the blocks is that call's integration. Device memory,
 *       4-byte aligned, owned by the caller, overwritten by each call.
 * block_spectra: a multiple of 64 in [64, 512] that divides n_spectra. INT8 with
 * CORR_FLAG_PLANAR only (CORR_EUNSUPPORTED otherwise). out = NULL switches the
 * output off. The extra bytes written are n_spectra / block_spectra times the
 * INT32 accumulator's size per call. */
CORR_API corr_status corr_set_short_time(corr_t *h, int32_t block_spectra, int32_t *out);

/* Cross-only X-engine: the rectangle of the visibility matrix between two input
 * ranges, V_ij = sum_a X_ai conj(X_aj) for i in [p0, p0 + n_p), j in [q0, q0 + n_q)
 * (Eq. 2 without the triangle restriction; two disjoint groups give the paper's
 * space-division node block, Section 4). One integration of chan_in, written to
 *   vis_out [n_chan][n_p][n_q]: complex int32 (2 x int32) for INT8, complex float
 *           otherwise; 8-byte aligned device memory, overwritten.
 * chan_in and gains as for corr_xengine (gains: g_i conj(g_j), float precisions).
 * The handle's accumulator and long integration are not touched. Runs on the
 * tensor-core X-engine (INT8, FP16, FP16_HILO; CORR_EUNSUPPORTED for FP32 and
 * CUDACORE). Ranges outside [0, n_in): CORR_EINVAL. */
CORR_API corr_status corr_xengine_cross(corr_t *h, const void *chan_in, const float *gains, int32_t p0,
                                        int32_t n_p, int32_t q0, int32_t n_q, void *vis_out, void *stream);

/* Copy the current integration accumulator to out: [n_chan][B] complex int32
 * (2 x int32) for INT8, complex float otherwise. Device pointer. */
CORR_API corr_status corr_get_accum(corr_t *h, void *out, void *stream);

/* Integration dump: vis64 += accumulator (FP64), accumulator = 0. If vis_out is
 * not NULL, the FP64 long-integration buffer is copied to it
 * ([n_chan][B] complex double, device). Asynchronous. The paper writes each
 * accumulation's visibilities out (Section 5, Section 6.3); the FP64 long
 * integration is this library's own addition, with no passage behind it.
 * On the INT8 and FP16_HILO tensor-core X-engine (without CORR_FLAG_FUSED_DUMP) a
 * dump with vis_out NULL is deferred: the finished accumulator is kept aside (the handle
 * then holds a second accumulator buffer, allocated on first use) and the next
 * corr_xengine launch adds it to the FP64 buffer from warps that would otherwise
 * idle, overlapping the X-engine. corr_flush, corr_dump with vis_out and
 * corr_fx_host complete a deferred dump first, so every reader of the FP64
 * buffer sees the same sums as with an immediate dump (bit for bit). */
CORR_API corr_status corr_dump(corr_t *h, double *vis_out, void *stream);

/* Complete any deferred dump (see corr_dump) on `stream` now: afterwards the FP64
 * long-integration buffer holds every dumped integration. No-op when none is
 * pending. (No counterpart in the paper.) */
CORR_API corr_status corr_flush(corr_t *h, void *stream);

/* Checkpoint / resume of the long integration: set the handle's FP64 buffer to
 *   vis_in [n_chan][B] complex double (device, 16-byte aligned; e.g. a buffer that
 *          corr_dump's vis_out filled earlier, in this process or another), or to
 *          zeros if vis_in is NULL.
 * The integration accumulator is cleared as by corr_dump (an integration in
 * progress is dropped), so the next X-engine call starts a new integration that
 * corr_dump adds to the restored buffer. Asynchronous on stream; the caller keeps
 * ownership of vis_in and may reuse it once the stream has passed this call.
 * Misaligned vis_in: CORR_EINVAL. */
CORR_API corr_status corr_restore_vis(corr_t *h, const double *vis_in, void *stream);

/* The whole step from host memory: raw voltages in, FP64 visibilities out, with
 * the host<->device copies pipelined against the kernels on two library-owned copy
 * streams (8 input blocks: copy-in overlaps the F-engine; 8 channel blocks:
 * X-engine and dump overlap the copy-out of the previous block).
 *   volt_host  [n_in][n_spectra * n_chan] complex int8, host (page-locked memory
 *              lets the copies run asynchronously)
 *   chan_scale [n_chan] float, device (see corr_fengine)
 *   vis_host   [n_chan][B] complex double, host: receives the FP64 long-integration
 *              buffer after this integration has been added to it (as corr_dump)
 * INT8 with CORR_FLAG_PLANAR only (CORR_EUNSUPPORTED otherwise). The first call
 * allocates two device copies of the inputs (successive calls fill them in turn)
 * and one of the channelised data. The results
 * are ordered on `stream`: the call's work is complete when `stream` reaches this
 * point. The copy-in of volt_host is not ordered after earlier work on `stream`: it
 * starts as soon as the F-engine of the call before the previous one has consumed
 * the device copy this call fills, so that back-to-back calls overlap one
 * integration's copy-in with the previous one's F-engine, X-engine and copy-out. volt_host must therefore hold the data when the call is
 * made and stay unchanged until `stream` reaches this point. */
CORR_API corr_status corr_fx_host(corr_t *h, const void *volt_host, const float *chan_scale, double *vis_host,
                                  void *stream);

/* The same whole step from host memory (Eqs. 1-2, Section 2), returning this
 * integration's exact visibilities instead of the long integration:
 *   acc_host [n_chan][B] complex int32 (2 x int32, Re then Im), host (page-locked
 *            memory lets the copies run asynchronously): the integration's sums,
 *            as corr_get_accum would give them; 8 bytes per visibility, half the
 *            FP64 copy of corr_fx_host.
 * The integration is also added to the FP64 long-integration buffer on the device
 * (as corr_dump), which stays there for corr_dump / corr_flush to read. Inputs,
 * ordering, the first call's allocations and the lifetime rule for volt_host are
 * those of corr_fx_host. INT8 with CORR_FLAG_PLANAR and without
 * CORR_FLAG_FUSED_DUMP (which keeps no INT32 accumulator): CORR_EUNSUPPORTED
 * otherwise; NULL pointers: CORR_EINVAL. */
CORR_API corr_status corr_fx_host_accum(corr_t *h, const void *volt_host, const float *chan_scale,
                                        int32_t *acc_host, void *stream);

/* Read and clear the handle's device status word. Returns CORR_ETIMEOUT (or
 * another CORR_* code) if a kernel of this handle gave up early since the last
 * check, CORR_OK otherwise. Synchronises `stream`. */
CORR_API corr_status corr_check_status(corr_t *h, void *stream);

/* Self-test of the failure detection every pipelined kernel relies on (its bounded
 * device-side waits): on `device`, one thread waits on an mbarrier that nothing
 * completes, with a time limit of limit_ns nanoseconds (1e6 .. 1e9). The wait must
 * give up after that limit, record CORR_ETIMEOUT in a device status word and return
 * instead of hanging; the barrier must then still complete on one arrival, and the
 * context stays usable. Synchronous. Returns CORR_OK when all of that happened,
 * CORR_ESTATE when the wait did not behave so, CORR_EINVAL for a limit out of range,
 * CORR_ECUDA on a CUDA error. */
CORR_API corr_status corr_selftest_bounded_wait(int32_t device, int64_t limit_ns);

/* Stages of the work a handle launches, for corr_stage_times (tracing; no
 * counterpart in the paper). */
enum {
    CORR_STAGE_FENGINE = 0,    /* F-engine FFT + re-packing + corner turn (k_fengine) */
    CORR_STAGE_PFB = 1,        /* polyphase filter bank FIR pass (k_pfb_fir) */
    CORR_STAGE_POWER = 2,      /* per-channel power pass */
    CORR_STAGE_PREP = 3,       /* conversion of the X-engine input to planar FP16 operands */
    CORR_STAGE_XENGINE = 4,    /* X-engine (triangle or rectangle) */
    CORR_STAGE_DUMP = 5,       /* integration dump into the FP64 long integration */
    CORR_STAGE_ADJ_PREP = 6,   /* adjoint: scale exponents and operand planes */
    CORR_STAGE_ADJ_GEMM = 7,   /* adjoint: the dX GEMM and its epilogue */
    CORR_STAGE_ADJ_REDUCE = 8, /* adjoint: fixed-order dL/dg reduction */
    CORR_STAGE_COUNT = 9
};

/* Per-stage timing of this handle's kernels (tracing). on != 0: every later call
 * brackets each stage's launches with a pair of CUDA events on the stream the
 * launches use (events are created on first use and kept); on == 0 stops
 * recording. Recording costs two event records per stage and call. */
CORR_API corr_status corr_set_stage_timing(corr_t *h, int32_t on);

/* Read and clear the timing since the last read: ms[CORR_STAGE_COUNT] receives
 * the summed event time per stage in milliseconds (overlapping stages on
 * different streams both count), launches[CORR_STAGE_COUNT] (or NULL) the number
 * of kernel launches per stage, counted whether or not timing is on. Waits for
 * the recorded events (host-synchronous). CORR_ESTATE if more than 65536 stage
 * records were made since the last read (the excess was not timed). */
CORR_API corr_status corr_stage_times(corr_t *h, double *ms, int64_t *launches);

/* Zero the accumulator and the FP64 long-integration buffer. */
CORR_API corr_status corr_reset(corr_t *h, void *stream);

/* Adjoint of corr_xengine (with gains) for gradient-based gain calibration. The
 * paper has no adjoint: this is the derivative of Eq. 2 with per-input gains
 * applied, for a loss over the visibilities, derived for this library.
 *   grad_vis  [n_chan][B] complex float: G_ij = dL/dV'_ij (PyTorch convention
 *             dL/dRe + j dL/dIm) of the gained visibilities, packed i >= j.
 *   chan_in   [n_chan][n_in][n_spectra] complex float: the forward input X.
 *   gains     [n_in] complex float, or NULL for unit gains.
 *   grad_chan [n_chan][n_in][n_spectra] complex float or NULL:
 *             dL/dX_f = diag(conj g) G^_f diag(g) X_f,
 *   grad_gains [n_in] complex float or NULL:
 *             dL/dg_m = sum_f sum_j G^_f,mj g_j V_f,jm,
 * with G^ the Hermitian completion of G (G^_ij = G_ij for i > j,
 * G^_ji = conj G_ij, G^_ii = 2 Re G_ii).
 * CORR_PREC_FP32: FP32 CUDA-core GEMM. CORR_PREC_FP16_HILO: the dX GEMM on tcgen05
 * tensor cores with both operands split into FP16 hi/lo parts; G^ diag(g) is scaled
 * per channel by an exact power of two into FP16 range, while chan_in is used as
 * given (its magnitudes should lie in FP16's normal range, 6.1e-5 .. 6.5e4, as for
 * the FP16 forward paths); needs n_in and n_spectra multiples of 8 (else
 * CORR_EUNSUPPORTED). Other precisions: CORR_ESTATE. dL/dg is summed in a fixed
 * order (bit-reproducible). The first call allocates the workspace. */
CORR_API corr_status corr_backward(corr_t *h, const float *grad_vis, const void *chan_in, const float *gains,
                          float *grad_chan, float *grad_gains, void *stream);

/* ---------------------------------------------------------------------------
 * Batched X-engine: many independent sub-arrays correlated (Eq. 2, INT8 exact)
 * by one persistent tensor-core launch that is captured once in a CUDA graph and
 * replayed. Inputs are planar FP16 int8 codes (the CORR_FLAG_PLANAR layout, e.g.
 * written by corr_fengine); outputs are INT32 pairs, overwritten by each run.
 * Pointers are fixed at create time: to process another window of data, write it
 * into the same buffers and run again.
 * ------------------------------------------------------------------------- */
typedef struct corr_batch_s corr_batch_t;

typedef struct corr_sub_desc {
    int32_t n_in;       /* inputs of the sub-array (1..65535) */
    int32_t n_chan;     /* channels */
    int32_t n_spectra;  /* spectra per integration: a multiple of 8, with n_spectra * 2 * 128^2 < 2^31 */
    int32_t reserved;   /* must be 0 */
    const void *planes; /* device, [n_chan][2][n_in][n_spectra] FP16 codes, 16-byte aligned */
    int32_t *vis;       /* device, [n_chan][n_in (n_in + 1) / 2][2] INT32, 8-byte aligned */
} corr_sub_desc;

/* Plan a batch: every (sub-array, channel, lower-triangle tile) work item is
 * spread over one CTA per SM, longest first. The descriptor array is copied; the
 * device buffers it names must outlive the batch.
 *   opts  NULL (INT8, current device) or precision CORR_PREC_INT8, xengine AUTO or
 *         TCGEN05, flags 0 or CORR_FLAG_PLANAR (the inputs are planar codes either
 *         way) and the device ordinal (-1: current); anything else is
 *         CORR_EUNSUPPORTED. Every later call on the batch runs on that device.
 * INT32 guard: each sub-array needs n_spectra * 2 * 128^2 < 2^31 (CORR_EOVERFLOW). */
CORR_API corr_status corr_batch_create(int32_t n_sub, const corr_sub_desc *subs, const corr_opts *opts,
                                       corr_batch_t **out);

/* Choose each sub-array's tile shape by timing: sub-arrays of <= 64 (<= 32)
 * inputs may pack 2 (up to 4) channels into one 128-row tensor-core tile. The
 * choices are read from / written to the JSON file cache_path (NULL: no cache)
 * keyed by (inputs, spectra), and the batch is re-planned. The timing runs are
 * queued on `stream` (so that they are ordered after the caller's writes of the
 * inputs), which this call synchronises; they overwrite the sub-arrays' outputs. */
CORR_API corr_status corr_batch_tune(corr_batch_t *b, const char *cache_path, void *stream);

/* Correlate every sub-array: one graph launch on `stream` (the graph is captured
 * on the first run after create or tune). */
CORR_API corr_status corr_batch_run(corr_batch_t *b, void *stream);

/* Read and clear the batch's device status word (CORR_ETIMEOUT if the kernel
 * gave up on a bounded wait). Synchronises stream. */
CORR_API corr_status corr_batch_check_status(corr_batch_t *b, void *stream);

/* Channels per tile chosen for sub-array `sub` (1, 2 or 4), -1 on bad arguments. */
CORR_API int32_t corr_batch_channels_per_tile(const corr_batch_t *b, int32_t sub);

CORR_API corr_status corr_batch_destroy(corr_batch_t *b);

#ifdef __cplusplus
}
#endif

#endif /* CORR_H */
