"""Seeded synthetic inputs for the FX correlator, shared by the CUDA path's tests,
the bench and the oracle's tests.

This module holds none of the correlator's arithmetic: it only draws random
voltages with the shapes and statistics of the workloads (noise plus delayed
point sources, int8 clipping, per-input gains, a point-source sky model). The
paper's own tests used synthetic 8-bit integer streams (Section 5); nothing here
reproduces a dataset.

Every array is drawn from numpy PCG64 streams keyed by
``SeedSequence(seed, spawn_key=(tag, index))``, one stream per input or per
channel, so any subset of channels or inputs can be regenerated on its own and
equals the same slice of the full array. Large arrays are filled by a thread
pool (numpy's generators release the GIL while filling).

Readings fixed here:
* "N(0,1)" complex noise: Re and Im each iid N(0, 1).
* point source of amplitude a: Re and Im of the common signal each iid N(0, a^2).
* raw int8 voltages: Re, Im = clip(rint(16 z + src), -127, 127) (symmetric clip).
* linear delays: s_i[t] = n_i[t] + p[t - d_i], p drawn for t in [-max_delay, K N).
* channelised sources: X_i[k, t] = n + sum_s p_s[k, t] exp(-j 2 pi k tau_si / N).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# stream tags
_T_NOISE, _T_SRC, _T_DELAY, _T_CHAN, _T_GAIN, _T_SUB, _T_SCALE = 1, 2, 3, 4, 5, 6, 7

CONFIGS = {
    # Plain FX, FP32: 16 antennas x 1 pol, 256-point FFT, 1024 spectra.
    "A": dict(n_ant=16, n_pol=1, n_chan=256, n_spectra=1024, precision="fp32"),
    # INT8 X-engine: 256 antennas x 2 pol, 1024 channels, 4096 spectra.
    "B": dict(n_ant=256, n_pol=2, n_chan=1024, n_spectra=4096, precision="int8"),
    # FP16: 1024 antennas x 2 pol, 4096 channels, 2048 spectra x 8 integrations.
    "C": dict(n_ant=1024, n_pol=2, n_chan=4096, n_spectra=2048, n_int=8, precision="fp16"),
    # Adjoint: 512 antennas x 1 pol, 1024 channels, 1024 spectra.
    "D": dict(n_ant=512, n_pol=1, n_chan=1024, n_spectra=1024, precision="fp32"),
    # Batched: 64 sub-arrays.
    "E": dict(n_sub=64, precision="int8"),
}


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=tuple(key))))


def _pool():
    return ThreadPoolExecutor(max_workers=max(1, min(32, os.cpu_count() or 1)))


def _normal_pair(rng: np.random.Generator, n: int, std: float) -> np.ndarray:
    """[n, 2] float32 of iid N(0, std^2)."""
    z = rng.standard_normal(2 * n, dtype=np.float32)
    if std != 1.0:
        z *= np.float32(std)
    return z.reshape(n, 2)


def _to_c64(pairs: np.ndarray) -> np.ndarray:
    return pairs.view(np.complex64).reshape(pairs.shape[:-1])


# --------------------------------------------------------------------------- raw voltages
def volt_fp32(n_in: int, n_chan: int, n_spectra: int, seed: int = 0, src_amp: float = 0.1,
              delays=None, noise: bool = True, circular: bool = False) -> np.ndarray:
    """Complex64 time series [n_in, n_spectra * n_chan]: N(0,1) noise plus a common
    point-source signal (Re, Im iid N(0, src_amp^2)) delayed by an integer number of
    samples per input (default d_i = i). ``circular`` delays the source within
    each N-sample frame (roll) instead of along the continuous stream; with
    ``noise=False`` that gives the noise-free exact phase-ramp case."""
    N, K = n_chan, n_spectra
    d = np.arange(n_in) if delays is None else np.asarray(delays, dtype=np.int64)
    max_d = int(d.max()) if d.size else 0
    rs = _rng(seed, _T_SRC, 0)
    if circular:
        p = _to_c64(_normal_pair(rs, K * N, src_amp)).reshape(K, N)
    else:
        p = _to_c64(_normal_pair(rs, K * N + max_d, src_amp))  # p[t] at index t + max_d
    out = np.empty((n_in, K * N), dtype=np.complex64)

    def fill(i):
        if circular:
            s = np.roll(p, int(d[i]), axis=1).reshape(-1)
        else:
            s = p[max_d - int(d[i]): max_d - int(d[i]) + K * N]
        if noise:
            out[i] = _to_c64(_normal_pair(_rng(seed, _T_NOISE, i), K * N, 1.0)) + s
        else:
            out[i] = s

    with _pool() as ex:
        list(ex.map(fill, range(n_in)))
    return out


def delays_int8(n_ant: int, seed: int = 0, max_delay: int = 15) -> np.ndarray:
    """Per-antenna integer delays, iid uniform on {0, ..., max_delay}."""
    return _rng(seed, _T_DELAY, 0).integers(0, max_delay + 1, size=n_ant)


def volt_int8(n_ant: int, n_pol: int, n_chan: int, n_spectra: int, seed: int = 0, sigma: float = 16.0,
              src_sigma: float = 1.6, max_delay: int = 15, lo: int = -127) -> np.ndarray:
    """Raw complex int8 voltages [n_in, n_spectra * n_chan, 2] (input i = ant * n_pol
    + pol): Re, Im = clip(rint(sigma z + src[t - d_ant]), lo, 127), src Re/Im iid
    N(0, src_sigma^2), d_ant uniform on {0..max_delay} shared by both pols. The
    workloads clip symmetrically (lo = -127); lo = -128 lets the edge tests reach
    the one int8 code whose negation is not an int8."""
    N, K = n_chan, n_spectra
    n_in = n_ant * n_pol
    d = delays_int8(n_ant, seed, max_delay)
    T = K * N
    src = _normal_pair(_rng(seed, _T_SRC, 0), T + max_delay, src_sigma)  # src[t] at t + max_delay
    out = np.empty((n_in, T, 2), dtype=np.int8)

    def fill(i):
        a = i // n_pol
        z = _normal_pair(_rng(seed, _T_NOISE, i), T, sigma)
        z += src[max_delay - int(d[a]): max_delay - int(d[a]) + T]
        np.rint(z, out=z)
        np.clip(z, float(lo), 127.0, out=z)
        out[i] = z.astype(np.int8)

    with _pool() as ex:
        list(ex.map(fill, range(n_in)))
    return out


# --------------------------------------------------------------------------- channelised data
def _chan_list(n_chan: int, chans):
    return list(range(n_chan)) if chans is None else [int(c) for c in chans]


def chan_int8(n_chan: int, n_in: int, n_spectra: int, seed: int = 0, chans=None,
              sigma: float = 16.0, lo: int = -127) -> np.ndarray:
    """Channelised complex int8 [n_sel, n_in, n_spectra, 2]: Re, Im =
    clip(rint(sigma z), lo, 127), one stream per channel (lo = -128 for the edge
    tests; the workloads use -127)."""
    cl = _chan_list(n_chan, chans)
    out = np.empty((len(cl), n_in, n_spectra, 2), dtype=np.int8)

    def fill(t):
        z = _normal_pair(_rng(seed, _T_CHAN, cl[t]), n_in * n_spectra, sigma)
        np.rint(z, out=z)
        np.clip(z, float(lo), 127.0, out=z)
        out[t] = z.reshape(n_in, n_spectra, 2).astype(np.int8)

    with _pool() as ex:
        list(ex.map(fill, range(len(cl))))
    return out


def source_params(n_src: int, n_in: int, seed: int = 0, tau_max: float = 64.0, flux=(0.5, 1.0)):
    """Per-(source, input) real delays tau ~ U[0, tau_max) samples and per-source
    fluxes A ~ U[flux]."""
    r = _rng(seed, _T_SRC, 1)
    tau = r.uniform(0.0, tau_max, size=(n_src, n_in))
    A = r.uniform(flux[0], flux[1], size=n_src)
    return tau, A


def chan_sources(n_chan: int, n_in: int, n_spectra: int, n_src: int, seed: int = 0, chans=None,
                 src_amp=None, flux=(0.5, 1.0), tau_max: float = 64.0) -> np.ndarray:
    """Channelised complex64 [n_sel, n_in, n_spectra]: N(0,1) noise plus n_src
    point sources. Source s in channel k has a common signal p_s[k, t]; input i
    sees it with the phase exp(-j 2 pi k tau_si / n_chan). With ``src_amp`` set,
    p_s has Re, Im iid N(0, src_amp^2); otherwise p_s = sqrt(A_s / 2)(z1 + j z2)
    with A_s the source flux, so E|p_s|^2 = A_s."""
    cl = _chan_list(n_chan, chans)
    tau, A = source_params(n_src, n_in, seed, tau_max, flux)
    out = np.empty((len(cl), n_in, n_spectra), dtype=np.complex64)

    def fill(t):
        k = cl[t]
        r = _rng(seed, _T_CHAN, k)
        x = _to_c64(_normal_pair(r, n_in * n_spectra, 1.0)).reshape(n_in, n_spectra).astype(np.complex128)
        for s in range(n_src):
            std = src_amp if src_amp is not None else math.sqrt(A[s] / 2.0)
            p = _to_c64(_normal_pair(r, n_spectra, std)).astype(np.complex128)
            ph = np.exp(-2j * np.pi * k * tau[s] / n_chan)  # [n_in]
            x += ph[:, None] * p[None, :]
        out[t] = x.astype(np.complex64)

    with _pool() as ex:
        list(ex.map(fill, range(len(cl))))
    return out


def gains(n_in: int, seed: int = 0, amp=(0.8, 1.2)) -> np.ndarray:
    """Per-input complex gains: |g| ~ U[amp], arg g ~ U[-pi, pi]."""
    r = _rng(seed, _T_GAIN, 0)
    mag = r.uniform(amp[0], amp[1], size=n_in)
    ph = r.uniform(-np.pi, np.pi, size=n_in)
    return (mag * np.exp(1j * ph)).astype(np.complex64)


def sky_model(n_chan: int, n_in: int, n_src: int, seed: int = 0, chans=None, tau_max: float = 64.0,
              flux=(0.5, 1.0), noise_power: float = 2.0) -> np.ndarray:
    """Point-source model visibilities [n_sel, B] (packed i >= j) matching
    ``chan_sources`` with flux-scaled sources: M_ij[k] = sum_s A_s exp(-j 2 pi k
    (tau_si - tau_sj) / N) for i > j and M_ii = sum_s A_s + noise_power."""
    cl = _chan_list(n_chan, chans)
    tau, A = source_params(n_src, n_in, seed, tau_max, flux)
    ii, jj = np.tril_indices(n_in)
    out = np.empty((len(cl), ii.size), dtype=np.complex128)
    for t, k in enumerate(cl):
        m = np.zeros(ii.size, dtype=np.complex128)
        for s in range(n_src):
            m += A[s] * np.exp(-2j * np.pi * k * (tau[s, ii] - tau[s, jj]) / n_chan)
        m[ii == jj] = A.sum() + noise_power
        out[t] = m
    return out


def weights(n_in: int, auto_weight: float = 0.0) -> np.ndarray:
    """w_ij = 1 for i > j and auto_weight on the autos, packed order."""
    ii, jj = np.tril_indices(n_in)
    return np.where(ii == jj, auto_weight, 1.0)


def subarrays(seed: int = 0, n_sub: int = 64, ant_range=(32, 2048), chan_choices=(256, 1024, 4096),
              spec_range=(512, 4096), spec_mult: int = 64):
    """Sub-array shapes for the batched workload: antennas log-uniform on
    ant_range (rounded), channels uniform from chan_choices, spectra uniform on
    spec_range rounded to a multiple of spec_mult; one pol."""
    r = _rng(seed, _T_SUB, 0)
    out = []
    for b in range(n_sub):
        m = int(round(math.exp(r.uniform(math.log(ant_range[0]), math.log(ant_range[1])))))
        c = int(chan_choices[int(r.integers(0, len(chan_choices)))])
        k = int(r.uniform(spec_range[0], spec_range[1]))
        k = max(spec_mult, int(round(k / spec_mult)) * spec_mult)
        out.append(dict(n_in=m, n_chan=c, n_spectra=k))
    return out
