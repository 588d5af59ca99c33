/*
 * FP64 CPU oracle for the FX correlator hot path (Wang & Harris 2013).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load it. It shares no code,
 * header, table or constant with the CUDA library and includes none of it.
 *
 * Every routine follows the definition in the paper directly, in double
 * precision, with no blocking or reordering beyond the plain loops:
 *   - oracle_dft_*  : Section 2, Eq. 1 (direct DFT, minus sign, no
 *                     normalisation, bins in natural order 0..N-1).
 *   - oracle_cmac_* : Section 2, Eq. 2 (cross-multiply-accumulate over the
 *                     A spectra of an integration), with the conjugate on the
 *                     second index: V_ij = sum_a S_{a,i} conj(S_{a,j}), i >= j,
 *                     which is conj(C_ij) of Eq. 2; autos included (Section 4,
 *                     the "triangle" of all non-redundant pairs).
 *
 * Packed lower-triangle index: b(i, j) = i (i + 1) / 2 + j for i >= j.
 * Complex data is interleaved (re, im).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* exp(-j 2 pi m / N) for m in [0, N): the Eq. 1 kernel, indexed by (k n) mod N
 * so that the argument of cos/sin never exceeds 2 pi. */
static double *twiddle_table(int32_t N) {
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!w) return NULL;
    for (int32_t m = 0; m < N; ++m) {
        double ang = 2.0 * M_PI * (double)m / (double)N;
        w[2 * m] = cos(ang);
        w[2 * m + 1] = -sin(ang);
    }
    return w;
}

/* One frame of Eq. 1 for the requested bins; x is the frame in double. */
static void dft_frame(const double *x, int32_t N, const double *w, const int32_t *bins, int32_t n_bins,
                      double *out) {
    for (int32_t b = 0; b < n_bins; ++b) {
        int64_t k = bins ? bins[b] : b;
        double sr = 0.0, si = 0.0;
        for (int32_t n = 0; n < N; ++n) {
            int64_t m = (k * n) % N;
            double xr = x[2 * n], xi = x[2 * n + 1];
            double wr = w[2 * m], wi = w[2 * m + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        out[2 * b] = sr;
        out[2 * b + 1] = si;
    }
}

/* Eq. 1 over n_frames consecutive frames of N complex samples.
 * in: [n_frames][N] complex; out: [n_frames][n_bins] complex double.
 * bins == NULL means all N bins (n_bins must then equal N). Returns 0 or -1. */
#define DEFINE_DFT(NAME, T)                                                                    \
    int NAME(const T *in, int64_t n_frames, int32_t N, const int32_t *bins, int32_t n_bins,    \
             double *out) {                                                                    \
        if (N <= 0 || n_bins <= 0 || (!bins && n_bins != N)) return -1;                        \
        double *w = twiddle_table(N);                                                          \
        if (!w) return -1;                                                                     \
        int err = 0;                                                                           \
        _Pragma("omp parallel")                                                                \
        {                                                                                      \
            double *x = (double *)malloc(sizeof(double) * 2 * (size_t)N);                      \
            if (!x) {                                                                          \
                _Pragma("omp atomic write") err = 1;                                           \
            } else {                                                                           \
                _Pragma("omp for schedule(static)")                                            \
                for (int64_t f = 0; f < n_frames; ++f) {                                       \
                    const T *src = in + 2 * (size_t)f * (size_t)N;                             \
                    for (int32_t n = 0; n < 2 * N; ++n) x[n] = (double)src[n];                 \
                    dft_frame(x, N, w, bins, n_bins, out + 2 * (size_t)f * (size_t)n_bins);    \
                }                                                                              \
                free(x);                                                                       \
            }                                                                                  \
        }                                                                                      \
        free(w);                                                                               \
        return err ? -1 : 0;                                                                   \
    }

DEFINE_DFT(oracle_dft_f64, double)
DEFINE_DFT(oracle_dft_f32, float)
DEFINE_DFT(oracle_dft_i8, int8_t)

/* Eq. 2 for n_chan independent channels.
 * X: [n_chan][n_in][K] complex; V: [n_chan][n_in (n_in + 1) / 2] complex.
 * Floating inputs accumulate in double; int8 inputs accumulate exactly in int64. */
#define DEFINE_CMAC(NAME, T, ACC)                                                              \
    void NAME(const T *X, int64_t n_chan, int32_t n_in, int64_t K, ACC *V) {                   \
        const int64_t B = (int64_t)n_in * (n_in + 1) / 2;                                      \
        _Pragma("omp parallel for collapse(2) schedule(dynamic, 1)")                           \
        for (int64_t c = 0; c < n_chan; ++c) {                                                 \
            for (int32_t i = 0; i < n_in; ++i) {                                               \
                const T *xi = X + 2 * ((size_t)c * n_in + i) * (size_t)K;                      \
                for (int32_t j = 0; j <= i; ++j) {                                             \
                    const T *xj = X + 2 * ((size_t)c * n_in + j) * (size_t)K;                  \
                    ACC re = 0, im = 0;                                                        \
                    for (int64_t a = 0; a < K; ++a) {                                          \
                        ACC ar = (ACC)xi[2 * a], ai = (ACC)xi[2 * a + 1];                      \
                        ACC br = (ACC)xj[2 * a], bi = (ACC)xj[2 * a + 1];                      \
                        /* x_i conj(x_j) */                                                    \
                        re += ar * br + ai * bi;                                               \
                        im += ai * br - ar * bi;                                               \
                    }                                                                          \
                    int64_t b = (int64_t)i * (i + 1) / 2 + j;                                  \
                    V[2 * (c * B + b)] = re;                                                   \
                    V[2 * (c * B + b) + 1] = im;                                               \
                }                                                                              \
            }                                                                                  \
        }                                                                                      \
    }

DEFINE_CMAC(oracle_cmac_f64, double, double)
DEFINE_CMAC(oracle_cmac_f32, float, double)
DEFINE_CMAC(oracle_cmac_i8, int8_t, int64_t)
