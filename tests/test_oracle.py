"""Pins for the FP64 oracle, each against something other than the oracle itself:
numpy's FFT and matmul, closed forms of Eq. 1 and Eq. 2, Parseval, Hermitian
symmetry, the delayed-source phase ramp, exact integer arithmetic, finite
differences, and the printed Eq. 3 instance. CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --------------------------------------------------------------------------- Eq. 1
@pytest.mark.parametrize("N", [1, 2, 3, 8, 17, 64, 256])
def test_dft_equals_numpy_fft(N):
    rng = np.random.default_rng(N)
    x = _crand(rng, 5, N)
    S = oracle.dft(x)
    ref = np.fft.fft(x, axis=-1)  # same sign, unnormalised
    assert np.max(np.abs(S - ref)) <= 1e-12 * N * max(1.0, np.max(np.abs(x)))


@pytest.mark.parametrize("N", [16, 256, 1024])
def test_dft_impulse_closed_form(N):
    m = N // 3 + 1
    x = np.zeros((1, N), complex)
    x[0, m] = 1.0
    S = oracle.dft(x)[0]
    k = np.arange(N)
    # exp(-j 2 pi k m / N), with k m reduced mod N so numpy's exp keeps full accuracy
    assert np.allclose(S, np.exp(-2j * np.pi * ((k * m) % N) / N), atol=1e-13, rtol=0)


def test_dft_constant_is_N_delta():
    N = 64
    x = np.full((1, N), 0.25 - 0.5j)
    S = oracle.dft(x)[0]
    want = np.zeros(N, complex)
    want[0] = N * (0.25 - 0.5j)
    assert np.max(np.abs(S - want)) < 1e-12


def test_dft_parseval_and_input_types():
    rng = np.random.default_rng(1)
    N = 128
    q = rng.integers(-127, 128, size=(6, N, 2)).astype(np.int8)
    xc = q[..., 0].astype(np.float64) + 1j * q[..., 1]
    S_i8 = oracle.dft(q)
    S_f32 = oracle.dft(xc.astype(np.complex64))
    S_f64 = oracle.dft(xc)
    assert np.array_equal(S_i8, S_f64)
    assert np.array_equal(S_f32, S_f64)  # int8 values are exact in float32
    lhs = np.sum(np.abs(S_f64) ** 2, axis=-1)
    rhs = N * np.sum(np.abs(xc) ** 2, axis=-1)
    assert np.allclose(lhs, rhs, rtol=1e-13)


def test_dft_bin_subset_and_channelise_layout():
    rng = np.random.default_rng(2)
    n_in, N, K = 3, 32, 4
    v = _crand(rng, n_in, K * N)
    bins = [0, 5, 31]
    S = oracle.channelise(v, N, bins)
    assert S.shape == (3, n_in, K)
    ref = np.fft.fft(v.reshape(n_in, K, N), axis=-1)[..., bins]  # [n_in, K, nb]
    assert np.allclose(S, np.transpose(ref, (2, 0, 1)), atol=1e-11)


# --------------------------------------------------------------------------- Eq. 2
def test_cmac_equals_matmul_lower_triangle():
    rng = np.random.default_rng(3)
    n_chan, n_in, K = 3, 7, 11
    X = _crand(rng, n_chan, n_in, K)
    V = oracle.cmac(X)
    full = X @ np.conj(np.transpose(X, (0, 2, 1)))  # V_ij = sum_a x_i conj x_j
    i, j = np.tril_indices(n_in)
    assert np.allclose(V, full[:, i, j], atol=1e-11)
    assert np.array_equal(oracle.packed_index(i, j), np.arange(i.size))


def test_cmac_int8_is_exact_integer():
    rng = np.random.default_rng(4)
    n_chan, n_in, K = 2, 9, 300
    q = rng.integers(-127, 128, size=(n_chan, n_in, K, 2)).astype(np.int8)
    q[0, 0, :, :] = 127  # extreme values
    q[0, 1, :, :] = -127
    V = oracle.cmac(q)
    a = q[..., 0].astype(np.int64)
    b = q[..., 1].astype(np.int64)
    i, j = np.tril_indices(n_in)
    re = np.einsum("cik,cjk->cij", a, a) + np.einsum("cik,cjk->cij", b, b)
    im = np.einsum("cik,cjk->cij", b, a) - np.einsum("cik,cjk->cij", a, b)
    assert V.dtype == np.int64
    assert np.array_equal(V[..., 0], re[:, i, j])
    assert np.array_equal(V[..., 1], im[:, i, j])


def test_cmac_hermitian_and_autos():
    rng = np.random.default_rng(5)
    n_in, K = 8, 16
    X = _crand(rng, 1, n_in, K)
    V = oracle.cmac(X)[0]
    # swapping the input order conjugates every cross product: V(j,i) = conj V(i,j)
    Vs = oracle.cmac(X[:, ::-1].copy())[0]
    for i in range(n_in):
        for j in range(i):
            a = V[oracle.packed_index(i, j)]
            b = Vs[oracle.packed_index(n_in - 1 - j, n_in - 1 - i)]
            assert abs(a - np.conj(b)) < 1e-12
    autos = V[oracle.packed_index(np.arange(n_in), np.arange(n_in))]
    assert np.all(autos.imag == 0.0)
    assert np.all(autos.real >= 0.0)


def test_autos_parseval_through_channeliser():
    """sum_k V_ii[k] = N sum_a sum_n |s_i[aN+n]|^2 (Eq. 1 + Eq. 2)."""
    rng = np.random.default_rng(6)
    n_in, N, K = 4, 32, 5
    v = _crand(rng, n_in, K * N)
    S = oracle.channelise(v, N)
    V = oracle.cmac(S)  # [N, B]
    autos = V[:, oracle.packed_index(np.arange(n_in), np.arange(n_in))].real.sum(axis=0)
    assert np.allclose(autos, N * np.sum(np.abs(v) ** 2, axis=1), rtol=1e-12)


def test_phase_ramp_circular_delay_exact():
    """Noise-free source delayed by d_i samples inside each frame:
    V_ij[k] = V_ii[k] exp(-j 2 pi k (d_i - d_j) / N) exactly, i.e. phase
    -2 pi f tau with f = k / N cycles/sample and tau = d_i - d_j."""
    N, K, n_in = 64, 6, 5
    d = np.array([0, 3, 7, 15, 1])
    v = synth.volt_fp32(n_in, N, K, seed=11, delays=d, noise=False, circular=True)
    V = oracle.cmac(oracle.channelise(v, N))
    k = np.arange(N)
    for i in range(n_in):
        vii = V[:, oracle.packed_index(i, i)]
        for j in range(i):
            want = vii * np.exp(-2j * np.pi * k * (d[i] - d[j]) / N)
            got = V[:, oracle.packed_index(i, j)]
            assert np.max(np.abs(got - want)) < 1e-9 * np.max(np.abs(vii))


def test_lag_spectrum_peaks_at_delay_config_A():
    """Config A (16 inputs, N=256, K=1024, linear delays d_i = i, source amplitude
    0.1 in unit noise): the lag spectrum |sum_k V_ij[k] e^{+j 2 pi k tau / N}| of
    every cross pair peaks at tau = d_i - d_j mod N."""
    c = synth.CONFIGS["A"]
    n_in, N, K = c["n_ant"] * c["n_pol"], c["n_chan"], c["n_spectra"]
    v = synth.volt_fp32(n_in, N, K, seed=0)
    V = oracle.cmac(oracle.channelise(v, N))  # [N, B]
    i, j = np.tril_indices(n_in)
    lag = np.abs(np.fft.ifft(V, axis=0))  # ifft carries e^{+j 2 pi k tau / N}
    peak = np.argmax(lag, axis=0)
    cross = i != j
    assert np.array_equal(peak[cross], ((i - j) % N)[cross])


# --------------------------------------------------------------------------- requant
def test_requant_rounding_and_clamp():
    x = np.array([2.5, 3.5, -2.5, -3.5, 0.49, 126.6, 127.49, 200.0, -200.0, -127.6, 0.0])
    S = (x + 1j * x[::-1]).reshape(1, 1, -1)
    q, margin = oracle.requant(S, np.array([1.0], np.float32))
    assert q[0, 0, :, 0].tolist() == [2, 4, -2, -4, 0, 127, 127, 127, -127, -127, 0]
    assert q[0, 0, :, 1].tolist() == list(reversed([2, 4, -2, -4, 0, 127, 127, 127, -127, -127, 0]))
    assert margin[0, 0, 0, 0] == 0.0 and margin[0, 0, 7, 0] == np.inf
    assert np.all(q >= -127)


def test_requant_scale_applied_per_channel():
    S = np.full((2, 1, 1), 10.0 + 0j)
    q, _ = oracle.requant(S, np.array([0.5, 2.0], np.float32))
    assert q[:, 0, 0, 0].tolist() == [5, 20]


def test_channel_power_parseval():
    rng = np.random.default_rng(7)
    n_in, N, K = 3, 16, 8
    v = _crand(rng, n_in, K * N)
    S = oracle.channelise(v, N)
    p = oracle.channel_power(S)
    total = np.sum(p) * 2 * n_in * K
    assert np.isclose(total, N * np.sum(np.abs(v) ** 2), rtol=1e-12)


# --------------------------------------------------------------------------- gains, dump
def test_gains_equal_correlating_gained_voltages():
    rng = np.random.default_rng(8)
    n_chan, n_in, K = 2, 6, 9
    X = _crand(rng, n_chan, n_in, K)
    g = _crand(rng, n_in)
    lhs = oracle.apply_gains(oracle.cmac(X), g, n_in)
    rhs = oracle.cmac(g[None, :, None] * X)
    assert np.allclose(lhs, rhs, atol=1e-11)


def test_dump_equals_one_long_integration():
    rng = np.random.default_rng(9)
    parts = [rng.integers(-127, 128, size=(2, 5, 8, 2)).astype(np.int8) for _ in range(3)]
    whole = np.concatenate(parts, axis=2)
    acc = oracle.dump([oracle.cmac(p) for p in parts])
    assert np.array_equal(acc, oracle.cmac(whole).astype(np.float64))


# --------------------------------------------------------------------------- calibration
@pytest.mark.parametrize("auto_w", [0.0, 1.0])
def test_gradients_match_central_differences(auto_w):
    rng = np.random.default_rng(10)
    n_chan, n_in, K = 3, 5, 7
    X = _crand(rng, n_chan, n_in, K)
    g = _crand(rng, n_in) * 0.7
    M = _crand(rng, n_chan, n_in * (n_in + 1) // 2)
    w = synth.weights(n_in, auto_w)
    L, dX, dg = oracle.loss_and_grads(X, g, M, w)
    h = 1e-6

    def Lg(gg):
        return oracle.loss(oracle.cmac(X), gg, M, w, K)

    for m in range(n_in):
        for unit in (1.0, 1j):
            gp, gm = g.copy(), g.copy()
            gp[m] += h * unit
            gm[m] -= h * unit
            fd = (Lg(gp) - Lg(gm)) / (2 * h)
            an = dg[m].real if unit == 1.0 else dg[m].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, np.max(np.abs(dg)))

    def LX(XX):
        return oracle.loss(oracle.cmac(XX), g, M, w, K)

    for (f, i, a) in [(0, 0, 0), (1, 3, 4), (2, 4, 6), (0, 2, 1)]:
        for unit in (1.0, 1j):
            Xp, Xm = X.copy(), X.copy()
            Xp[f, i, a] += h * unit
            Xm[f, i, a] -= h * unit
            fd = (LX(Xp) - LX(Xm)) / (2 * h)
            an = dX[f, i, a].real if unit == 1.0 else dX[f, i, a].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, np.max(np.abs(dX)))


def test_loss_zero_at_model():
    n_chan, n_in, K = 2, 4, 3
    rng = np.random.default_rng(12)
    X = _crand(rng, n_chan, n_in, K)
    g = _crand(rng, n_in)
    M = oracle.apply_gains(oracle.cmac(X), g, n_in) / K
    L, dX, dg = oracle.loss_and_grads(X, g, M, synth.weights(n_in, 1.0))
    assert L < 1e-20 and np.max(np.abs(dg)) < 1e-9 and np.max(np.abs(dX)) < 1e-9


# --------------------------------------------------------------------------- golden
def test_golden_eq3_triangle_count():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eq3_triangle_count.txt")) if l.strip() and l[0] != "#"]
    for ns, nc in rows:
        ns, nc = int(ns), int(nc)
        assert oracle.n_baselines(ns) == nc
        assert (math.isqrt(8 * nc + 1) - 1) // 2 == ns
        i, j = oracle.tri_pairs(ns)
        assert i.size == nc and np.all(i >= j)


# --------------------------------------------------------------------------- delay compensation
def test_delay_split_rounding():
    D, f = oracle.delay_split(np.array([0.0, 2.4, 2.5, -2.5, 3.75, -0.2], np.float32))
    assert D.tolist() == [0, 2, 3, -3, 4, 0]
    assert np.allclose(f, [0.0, 0.4, -0.5, 0.5, -0.25, -0.2], atol=1e-6)


def test_delay_zero_is_plain_channelise():
    v = synth.volt_fp32(3, 64, 5, seed=2)
    assert np.array_equal(oracle.channelise_delayed(v, 64, np.zeros(3)), oracle.channelise(v, 64))
    vi = synth.volt_int8(2, 1, 16, 7, seed=3)
    assert np.array_equal(oracle.channelise_delayed(vi, 16, np.zeros(2)), oracle.channelise(vi, 16))


def test_delay_tone_closed_form():
    """A tone at bin k0 delayed by tau: exp(j 2 pi k0 (t - tau) / N). Uncompensated,
    its bin-k0 value is N exp(-j 2 pi k0 tau / N); compensated it is N (zero phase)
    in every frame whose advanced samples lie inside the record, and the other bins
    stay empty."""
    N, K, k0 = 64, 6, 5
    tau = np.array([0.0, 3.3, -2.7, 70.25], np.float32)
    t = np.arange(K * N)
    taud = tau.astype(np.float64)
    v = np.exp(2j * np.pi * k0 * (t[None, :] - taud[:, None]) / N)
    S0 = oracle.channelise(v, N)
    assert np.allclose(S0[k0], N * np.exp(-2j * np.pi * k0 * taud / N)[:, None], atol=1e-9 * N)
    S = oracle.channelise_delayed(v, N, tau)
    D, _ = oracle.delay_split(tau)
    for i in range(len(tau)):
        a_lo = int(np.ceil(max(0, -D[i]) / N))
        a_hi = K - int(np.ceil(max(0, D[i]) / N))
        assert a_hi > a_lo
        assert np.allclose(S[k0, i, a_lo:a_hi], N, atol=1e-9 * N), i
        others = np.delete(S[:, i, a_lo:a_hi], k0, axis=0)
        assert np.max(np.abs(others)) <= 1e-9 * N


def test_delay_integer_advance_recovers_source():
    """Inputs that carry one stream p delayed by whole samples (s_i[t] = p[t - D_i],
    zero before the stream starts) are re-aligned exactly: every frame whose advanced
    samples are recorded equals the frame of p, bit for bit."""
    N, K = 16, 9
    rng = np.random.default_rng(5)
    p = rng.standard_normal(K * N) + 1j * rng.standard_normal(K * N)
    D = np.array([0, 5, 17, 32])
    v = np.zeros((len(D), K * N), np.complex128)
    for i, d in enumerate(D):
        v[i, d:] = p[: K * N - d]
    S = oracle.channelise_delayed(v, N, D.astype(np.float32))
    P = oracle.channelise(p[None, :], N)[:, 0, :]
    for i, d in enumerate(D):
        a_hi = K - int(np.ceil(d / N))
        assert np.array_equal(S[:, i, :a_hi], P[:, :a_hi]), i
        assert np.all(S[:, i, a_hi:] != P[:, a_hi:]) or a_hi == K


# --------------------------------------------------------------------------- polyphase filter bank
def _sinc_hann(P, N):
    x = (np.arange(P * N) - P * N / 2 + 0.5) / N
    return (np.sinc(x) * np.hanning(P * N)).reshape(P, N).astype(np.float32)


def test_pfb_single_unit_tap_is_channelise():
    v = synth.volt_fp32(3, 64, 7, seed=4)
    S = oracle.channelise_pfb(v, 64, np.ones((1, 64), np.float32))
    assert np.allclose(S, oracle.channelise(v, 64), rtol=0, atol=1e-12 * np.abs(S).max())


def test_pfb_single_tap_is_windowed_dft():
    N, K = 32, 6
    v = synth.volt_fp32(2, N, K, seed=6)
    w = np.random.default_rng(1).uniform(0.2, 1.0, N).astype(np.float32)
    S = oracle.channelise_pfb(v, N, w[None, :])
    frames = v.reshape(2, K, N).astype(np.complex128) * w.astype(np.float64)[None, None, :]
    ref = np.transpose(np.fft.fft(frames, axis=-1), (2, 0, 1))
    assert np.allclose(S, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_pfb_tone_closed_form():
    """A tone at bin k0: every full frame sum is exp(j 2 pi k0 n / N) H[n] with
    H[n] = sum_p h[p][n], so S[k] = sum_n H[n] exp(-j 2 pi (k - k0) n / N)."""
    N, K, P, k0 = 64, 9, 4, 11
    h = _sinc_hann(P, N)
    t = np.arange(K * N)
    v = np.exp(2j * np.pi * k0 * t / N)[None, :]
    S = oracle.channelise_pfb(v, N, h)[:, 0, :]
    H = h.astype(np.float64).sum(axis=0)
    want = np.fft.fft(H)[(np.arange(N) - k0) % N]
    full = K - P + 1
    assert np.allclose(S[:, :full], want[:, None], rtol=0, atol=1e-9 * np.abs(want).max())


def test_pfb_brute_force_tiny():
    """Direct double sum over taps and samples, pure Python, on a tiny case with
    delays (integer advance, zero fill past the record, per-channel phase)."""
    N, K, P = 8, 5, 3
    rng = np.random.default_rng(2)
    v = (rng.standard_normal((2, K * N)) + 1j * rng.standard_normal((2, K * N))).astype(np.complex64)
    h = rng.uniform(-1, 1, (P, N)).astype(np.float32)
    tau = np.array([2.25, -9.5], np.float32)
    S = oracle.channelise_pfb(v, N, h, delays=tau)
    D, f = oracle.delay_split(tau)
    for i in range(2):
        for a in range(K):
            for k in range(N):
                acc = 0j
                for n in range(N):
                    y = 0j
                    for p in range(P):
                        tt = (a + p) * N + n + int(D[i])
                        if 0 <= tt < K * N:
                            y += float(h[p, n]) * complex(v[i, tt])
                    acc += y * np.exp(-2j * np.pi * k * n / N)
                acc *= np.exp(2j * np.pi * k * f[i] / N)
                assert abs(S[k, i, a] - acc) <= 1e-9 * (1 + abs(acc))
