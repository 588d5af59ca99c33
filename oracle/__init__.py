"""FP64 CPU oracle for the FX correlator hot path (Wang & Harris 2013).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs may
import it. It shares no code with the CUDA library (``paper_1305_5639_gb300``)
and imports nothing from it; the two meet only in the seeded input generators
of ``synth``.

What each function follows:

* ``dft``            -- Section 2, Eq. 1: S[k] = sum_n s[n] exp(-j 2 pi k n / N),
                        unnormalised, natural bin order, direct evaluation in C.
* ``cmac``           -- Section 2, Eq. 2 with the conjugate on the second index
                        (V_ij = sum_a S_ai conj(S_aj) = conj(C_ij)), i >= j packed,
                        autos included (Section 4, "triangle" X-engine). Triple
                        loop in C; int8 input accumulates exactly in int64.
* ``requant``        -- 8-bit re-packing of the spectra (Section 5: all data is
                        carried in 8-bit integers; Section 6.2: the FFT expands the
                        data, so it is packed again). Decision taken in FP32.
* ``apply_gains``    -- per-input complex gain model V'_ij = g_i conj(g_j) V_ij.
* ``dump``           -- long integration: sum of per-integration visibilities.
* ``loss_and_grads`` -- weighted least-squares calibration loss and its analytic
                        gradient (PyTorch convention dL/dRe + j dL/dIm).
* ``channel_power``  -- per-channel mean power per real component of the spectra.
* ``channelise_pfb`` -- polyphase filter-bank front end ahead of Eq. 1 (the
                        windowed multi-tap channeliser the paper's F-engine does
                        not use, Section 5 / Section 7): each frame is the
                        tap-weighted sum of n_taps consecutive frames, then Eq. 1.
* ``channelise_delayed`` -- delay compensation ahead of Eq. 1 (a station-based
                        function the paper leaves for future work, Section 7):
                        integer-sample advance of each input's stream, Eq. 1 on the
                        shifted frames, then a per-channel phase for the fractional
                        remainder.

Pins (tests/test_oracle.py) tie every function to something outside itself:
numpy's FFT, closed forms (impulse, constant, delayed source), Parseval, Hermitian
symmetry, brute force via numpy matmul, finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP over frames/channels)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            for name in ("oracle_dft_f64", "oracle_dft_f32", "oracle_dft_i8"):
                fn = getattr(lib, name)
                fn.argtypes = [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int32, P]
                fn.restype = ctypes.c_int
            for name in ("oracle_cmac_f64", "oracle_cmac_f32", "oracle_cmac_i8"):
                fn = getattr(lib, name)
                fn.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, P]
                fn.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- indices
def n_baselines(n_in: int) -> int:
    """Number of packed pairs i >= j, autos included: n (n + 1) / 2 (the same count
    as Eq. 3's correlation nodes for n_s streaming nodes, Section 4.1)."""
    return n_in * (n_in + 1) // 2


def packed_index(i, j):
    """b(i, j) = i (i + 1) / 2 + j for i >= j."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * (i + 1) // 2 + j


def tri_pairs(n_in: int):
    """(i, j) arrays of all packed pairs in packed order."""
    i, j = np.tril_indices(n_in)
    return i.astype(np.int64), j.astype(np.int64)


# --------------------------------------------------------------------------- Eq. 1
def dft(frames: np.ndarray, bins=None) -> np.ndarray:
    """Eq. 1 on each frame: frames [..., N] complex (complex128/complex64) or
    [..., N, 2] int8 (re, im). Returns complex128 [..., n_bins]."""
    lib = _load()
    if frames.dtype == np.int8:
        assert frames.shape[-1] == 2
        N = frames.shape[-2]
        lead = frames.shape[:-2]
        src = np.ascontiguousarray(frames)
        fn = lib.oracle_dft_i8
    elif frames.dtype == np.complex64:
        N = frames.shape[-1]
        lead = frames.shape[:-1]
        src = np.ascontiguousarray(frames)
        fn = lib.oracle_dft_f32
    else:
        N = frames.shape[-1]
        lead = frames.shape[:-1]
        src = np.ascontiguousarray(frames, dtype=np.complex128)
        fn = lib.oracle_dft_f64
    n_frames = int(np.prod(lead)) if lead else 1
    if bins is None:
        b = None
        n_bins = N
    else:
        b = np.ascontiguousarray(np.asarray(bins, dtype=np.int32))
        assert np.all((b >= 0) & (b < N))
        n_bins = int(b.size)
    out = np.empty(tuple(lead) + (n_bins,), dtype=np.complex128)
    rc = fn(_ptr(src), n_frames, N, None if b is None else _ptr(b), n_bins, _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle_dft failed")
    return out


def channelise(volt: np.ndarray, N: int, bins=None) -> np.ndarray:
    """Split each input's time series into consecutive N-sample frames (spectrum a
    covers samples aN .. aN+N-1) and apply Eq. 1. volt: [n_in, K*N] complex or
    [n_in, K*N, 2] int8. Returns [n_bins, n_in, K] complex128 (channel-major)."""
    n_in = volt.shape[0]
    if volt.dtype == np.int8:
        K = volt.shape[1] // N
        frames = volt.reshape(n_in, K, N, 2)
    else:
        K = volt.shape[1] // N
        frames = volt.reshape(n_in, K, N)
    S = dft(frames, bins)  # [n_in, K, n_bins]
    return np.ascontiguousarray(np.transpose(S, (2, 0, 1)))


# --------------------------------------------------------------------------- delay compensation
def delay_split(delays: np.ndarray):
    """tau_i (samples) -> (D_i, f_i): D_i the nearest integer (halves rounded away
    from zero), f_i = tau_i - D_i in [-0.5, 0.5]. The split is decided on the FP32
    value, the precision in which delays are handed over."""
    t = np.asarray(delays, dtype=np.float32).astype(np.float64)
    D = np.where(t >= 0, np.floor(t + 0.5), -np.floor(-t + 0.5)).astype(np.int64)
    return D, t - D


def channelise_delayed(volt: np.ndarray, N: int, delays: np.ndarray, bins=None) -> np.ndarray:
    """Delay-compensated channelisation. Input i's stream s_i, delayed by tau_i
    samples, is advanced by its integer part: s'_i[t] = s_i[t + D_i] (zero where
    t + D_i falls outside the recorded K*N samples); each N-sample frame goes
    through Eq. 1; channel k is multiplied by exp(+j 2 pi k f_i / N) for the
    fractional remainder f_i (k the natural bin index 0..N-1). A delayed tone at a
    bin frequency comes out with zero phase. Returns [n_bins, n_in, K] complex128."""
    n_in = volt.shape[0]
    D, f = delay_split(delays)
    L = volt.shape[1]
    shifted = np.zeros_like(volt)
    for i in range(n_in):
        d = int(D[i])
        lo, hi = max(0, -d), min(L, L - d)  # t with 0 <= t + d < L
        if hi > lo:
            shifted[i, lo:hi] = volt[i, lo + d:hi + d]
    S = channelise(shifted, N, bins)
    k = np.arange(N, dtype=np.float64) if bins is None else np.asarray(bins, dtype=np.float64)
    ph = np.exp(2j * np.pi * np.outer(k, f) / N)  # [n_bins, n_in]
    return S * ph[:, :, None]


# --------------------------------------------------------------------------- polyphase filter bank
def channelise_pfb(volt: np.ndarray, N: int, window: np.ndarray, delays=None, bins=None) -> np.ndarray:
    """Polyphase filter-bank channelisation. window: [n_taps, N] real weights h[p][n].
    Spectrum a of input i is Eq. 1 applied to the frame
        y_a[n] = sum_{p < n_taps} h[p][n] s'_i[(a + p) N + n],   n < N,
    where s'_i[t] = s_i[t + D_i] is the input's stream advanced by its integer delay
    (D_i = 0 without `delays`), zero wherever t + D_i is not one of the K*N recorded
    samples, so every input keeps K spectra; with `delays` channel k is then
    multiplied by exp(+j 2 pi k f_i / N), as in channelise_delayed.
    Returns [n_bins, n_in, K] complex128."""
    h = np.asarray(window, dtype=np.float32).astype(np.float64)
    P = h.shape[0]
    assert h.shape == (P, N)
    n_in = volt.shape[0]
    if volt.dtype == np.int8:
        s = volt[..., 0].astype(np.float64) + 1j * volt[..., 1].astype(np.float64)
    else:
        s = volt.astype(np.complex128)
    L = s.shape[1]
    K = L // N
    Lp = L + (P - 1) * N  # the frames of the last spectra reach past the record
    D, f = delay_split(np.zeros(n_in) if delays is None else delays)
    # s'_i[t] = s_i[t + D_i] for t < Lp, zero where t + D_i is not a recorded sample
    padded = np.zeros((n_in, Lp), np.complex128)
    for i in range(n_in):
        d = int(D[i])
        lo, hi = max(0, -d), min(Lp, L - d)
        if hi > lo:
            padded[i, lo:hi] = s[i, lo + d:hi + d]
    frames = np.zeros((n_in, K, N), np.complex128)
    for p in range(P):  # frame a takes frames a .. a + P - 1 of the stream
        frames += h[p][None, None, :] * padded[:, p * N: p * N + K * N].reshape(n_in, K, N)
    S = np.ascontiguousarray(np.transpose(dft(frames, bins), (2, 0, 1)))
    k = np.arange(N, dtype=np.float64) if bins is None else np.asarray(bins, dtype=np.float64)
    return S * np.exp(2j * np.pi * np.outer(k, f) / N)[:, :, None]


# --------------------------------------------------------------------------- requant
def requant(S: np.ndarray, scale: np.ndarray):
    """8-bit re-packing of spectra S [n_chan, n_in, K] (complex) with one FP32
    scale per channel. Each of Re and Im: v = fl32(fl32(x) * scale_k), clamped to
    [-127, 127] and rounded half-to-even -- the decision taken in FP32, the
    precision of the channeliser. Symmetric clipping keeps -q representable.

    Returns (q [n_chan, n_in, K, 2] int8, margin [n_chan, n_in, K, 2] float64),
    where margin is the FP64 distance of x*scale_k from the nearest rounding
    boundary (k + 0.5), used to decide which codes are unique."""
    scale = np.asarray(scale, dtype=np.float32)
    parts = np.stack([S.real, S.imag], axis=-1)  # float64
    sc = scale.reshape((-1,) + (1,) * (parts.ndim - 1))
    v32 = (parts.astype(np.float32) * sc).astype(np.float32)
    v32 = np.clip(v32, np.float32(-127.0), np.float32(127.0))
    q = np.rint(v32).astype(np.int8)  # numpy rint: round half to even
    v64 = parts * sc.astype(np.float64)
    margin = np.abs(np.abs(v64 - np.floor(v64)) - 0.5)
    # clamped values are unique whatever the rounding
    margin = np.where(np.abs(v64) > 127.5, np.inf, margin)
    return q, margin


def channel_power(S: np.ndarray) -> np.ndarray:
    """Mean power per real component of each channel: sum(|S|^2) / (2 n_in K).
    S: [n_chan, n_in, K] complex. Its square root is the per-component RMS."""
    p = (S.real.astype(np.float64) ** 2 + S.imag.astype(np.float64) ** 2)
    return p.sum(axis=(1, 2)) / (2.0 * S.shape[1] * S.shape[2])


# --------------------------------------------------------------------------- Eq. 2
def cmac(X: np.ndarray) -> np.ndarray:
    """Eq. 2 (conjugate on the second index) per channel, triple loop in C.
    X: [n_chan, n_in, K] complex, or [n_chan, n_in, K, 2] int8.
    Returns [n_chan, B] complex128, or [n_chan, B, 2] int64 for int8 input."""
    lib = _load()
    if X.dtype == np.int8:
        n_chan, n_in, K, two = X.shape
        assert two == 2
        src = np.ascontiguousarray(X)
        V = np.empty((n_chan, n_baselines(n_in), 2), dtype=np.int64)
        lib.oracle_cmac_i8(_ptr(src), n_chan, n_in, K, _ptr(V))
        return V
    n_chan, n_in, K = X.shape
    if X.dtype == np.complex64:
        src = np.ascontiguousarray(X)
        fn = lib.oracle_cmac_f32
    else:
        src = np.ascontiguousarray(X, dtype=np.complex128)
        fn = lib.oracle_cmac_f64
    V = np.empty((n_chan, n_baselines(n_in)), dtype=np.complex128)
    fn(_ptr(src), n_chan, n_in, K, _ptr(V))
    return V


def unpack_full(Vp: np.ndarray, n_in: int) -> np.ndarray:
    """Packed lower triangle [..., B] -> full Hermitian [..., n_in, n_in]
    (upper triangle filled by V_ji = conj V_ij)."""
    i, j = tri_pairs(n_in)
    full = np.zeros(Vp.shape[:-1] + (n_in, n_in), dtype=np.complex128)
    full[..., i, j] = Vp
    full[..., j, i] = np.conj(Vp)
    return full


# --------------------------------------------------------------------------- gains, dump
def apply_gains(Vp: np.ndarray, g: np.ndarray, n_in: int) -> np.ndarray:
    """V'_ij = g_i conj(g_j) V_ij on packed visibilities [..., B]."""
    i, j = tri_pairs(n_in)
    g = np.asarray(g, dtype=np.complex128)
    return Vp * (g[i] * np.conj(g[j]))


def dump(integrations) -> np.ndarray:
    """Long integration: FP64 sum of per-integration visibilities."""
    acc = None
    for V in integrations:
        V = np.asarray(V)
        V = V.astype(np.complex128) if np.iscomplexobj(V) else V.astype(np.float64)
        acc = V.copy() if acc is None else acc + V
    return acc


# --------------------------------------------------------------------------- calibration
def hermitian_complete(Gp: np.ndarray, n_in: int) -> np.ndarray:
    """Packed G (i >= j) -> full G_hat: G_hat_ij = G_ij (i > j),
    G_hat_ji = conj G_ij, G_hat_ii = 2 Re G_ii."""
    i, j = tri_pairs(n_in)
    full = np.zeros(Gp.shape[:-1] + (n_in, n_in), dtype=np.complex128)
    off = i != j
    full[..., i[off], j[off]] = Gp[..., off]
    full[..., j[off], i[off]] = np.conj(Gp[..., off])
    d = ~off
    full[..., i[d], i[d]] = 2.0 * Gp[..., d].real
    return full


def loss(Vraw: np.ndarray, g: np.ndarray, M: np.ndarray, w: np.ndarray, K: int) -> float:
    """L = sum_f sum_{i>=j} w_ij |g_i conj(g_j) V_f,ij / K - M_f,ij|^2.
    Vraw: [n_chan, B] raw (ungained) visibilities; M: [n_chan, B]; w: [B]."""
    n_in = len(g)
    R = apply_gains(Vraw, g, n_in) / K - M
    return float(np.sum(w * (R.real ** 2 + R.imag ** 2)))


def loss_and_grads(X: np.ndarray, g: np.ndarray, M: np.ndarray, w: np.ndarray, Vraw=None):
    """Loss above plus its gradient (PyTorch convention grad = dL/dRe + j dL/dIm).

    With R = V'/K - M and G_ij = 2 w_ij R_ij / K (i >= j, the gradient of L with
    respect to V'_ij), and G_hat its Hermitian completion:
        dL/dg_m  = sum_f sum_j G_hat_f,mj g_j V_f,jm
        dL/dX_f  = diag(conj g) G_hat_f diag(g) X_f
    X: [n_chan, n_in, K] complex. Returns (L, dX [n_chan, n_in, K], dg [n_in])."""
    n_chan, n_in, K = X.shape
    g = np.asarray(g, dtype=np.complex128)
    if Vraw is None:
        Vraw = cmac(X)
    R = apply_gains(Vraw, g, n_in) / K - M
    L = float(np.sum(w * (R.real ** 2 + R.imag ** 2)))
    G = 2.0 * w * R / K
    Gh = hermitian_complete(G, n_in)  # [n_chan, n_in, n_in]
    Vf = unpack_full(Vraw, n_in)  # [n_chan, n_in, n_in], Vf[f, a, b] = V_ab
    # dg_m = sum_f sum_j Gh[f, m, j] g_j V[f, j, m]
    dg = np.einsum("fmj,j,fjm->m", Gh, g, Vf)
    P = np.conj(g)[None, :, None] * Gh * g[None, None, :]
    dX = np.matmul(P, X.astype(np.complex128))
    return L, dX, dg
