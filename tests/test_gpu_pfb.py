"""Polyphase filter-bank front end of the F-engine against the oracle's direct
definition (tap-weighted frame sums, Eq. 1), alone and with delay compensation."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _sinc_hann(P, N):
    x = (np.arange(P * N) - P * N / 2 + 0.5) / N
    return (np.sinc(x) * np.hanning(P * N)).reshape(P, N).astype(np.float32)


@pytest.mark.parametrize("N,n_in,K,P,with_delays", [(16, 3, 21, 4, False), (64, 2, 9, 3, True),
                                                     (256, 3, 13, 4, False), (1024, 2, 11, 4, True),
                                                     (1024, 1, 6, 1, False), (512, 2, 7, 4, True),
                                                     (2048, 1, 5, 3, True)])
def test_pfb_fp32_matches_oracle(cuda_ok, N, n_in, K, P, with_delays):
    v = synth.volt_fp32(n_in, N, K, seed=N + P)
    h = _sinc_hann(P, N)
    d = np.random.default_rng(N).uniform(-1.2 * N, 1.2 * N, n_in).astype(np.float32) if with_delays else None
    c = api.Correlator(n_in, 1, N, K, precision="fp32")
    c.set_pfb(h)
    if with_delays:
        c.set_delays(d)
    S = c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy().astype(np.complex128)
    ref = oracle.channelise_pfb(v, N, h, delays=d)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(S - ref)) <= 2e-5 * rms
    c.set_pfb(None)  # off again: the plain channeliser
    if with_delays:
        c.set_delays(None)
    S0 = c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(S0 - oracle.channelise(v, N))) <= 1e-5 * np.sqrt(np.mean(np.abs(S0) ** 2))
    c.close()


@pytest.mark.parametrize("planar", [False, True])
def test_pfb_int8_requant(cuda_ok, planar):
    N, n_ant, n_pol, K, P = 256, 2, 2, 24, 4
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=17)
    h = _sinc_hann(P, N)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=planar)
    c.set_pfb(h)
    S = oracle.channelise_pfb(v, N, h)
    scale = (16.0 / np.sqrt(np.mean(np.abs(S) ** 2, axis=(1, 2)) / 2)).astype(np.float32)
    out = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    if planar:
        out = np.transpose(out, (0, 2, 3, 1)).astype(np.int8)
    q, margin = oracle.requant(S, scale)
    eps = 8 * np.log2(N) * P * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 8
    sure = margin > eps
    assert np.array_equal(out[sure], q[sure])
    assert np.all(np.abs(out.astype(np.int32) - q.astype(np.int32)) <= 1)
    # the power pass sees the filter bank too
    p = c.fengine_power(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.allclose(p, oracle.channel_power(S), rtol=1e-4)
    c.close()


@pytest.mark.parametrize("N,n_ant,K,P,with_delays,planar", [(1024, 2, 16, 3, True, True), (256, 3, 21, 5, True, False),
                                                              (64, 2, 24, 8, False, True), (16, 2, 30, 1, True, False)])
def test_pfb_int8_fused_taps_and_delays(cuda_ok, N, n_ant, K, P, with_delays, planar):
    """int8 voltages through the filter bank and the re-packing: tap counts that are
    not a multiple of 4, delays (advance past both ends of the record, fractional
    phase) and both output layouts against the oracle's definition."""
    n_pol = 2
    n_in = n_ant * n_pol
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=N + P)
    h = _sinc_hann(P, N)
    d = None
    if with_delays:
        d = np.random.default_rng(P).uniform(-1.5 * N, 1.5 * N, n_in).astype(np.float32)
        d[0] = 0.0
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=planar)
    c.set_pfb(h)
    if with_delays:
        c.set_delays(d)
    S = oracle.channelise_pfb(v, N, h, delays=d)
    scale = (16.0 / np.sqrt(np.mean(np.abs(S) ** 2, axis=(1, 2)) / 2)).astype(np.float32)
    out = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    if planar:
        out = np.transpose(out, (0, 2, 3, 1)).astype(np.int8)
    q, margin = oracle.requant(S, scale)
    eps = 8 * np.log2(N) * max(P, 2) * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 8
    sure = margin > eps
    assert sure.mean() > 0.9
    assert np.array_equal(out[sure], q[sure])
    assert np.all(np.abs(out.astype(np.int32) - q.astype(np.int32)) <= 1)
    p_gpu = c.fengine_power(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.allclose(p_gpu, oracle.channel_power(S), rtol=1e-4)
    c.close()


def test_pfb_tone_leakage(cuda_ok):
    """A tone halfway between two bins leaks far less into distant channels through
    the 4-tap filter bank than through the plain FFT (the filter bank's purpose),
    and the GPU agrees with the oracle on both."""
    N, K, P = 256, 16, 4
    t = np.arange(K * N)
    v = np.exp(2j * np.pi * 40.5 * t / N)[None, :].astype(np.complex64)
    c = api.Correlator(1, 1, N, K, precision="fp32")
    plain = np.abs(c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy()[:, 0, 4])
    c.set_pfb(_sinc_hann(P, N))
    pfb = np.abs(c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy()[:, 0, 4])
    far = np.r_[0:30, 51:N]
    assert pfb[far].max() / pfb.max() < 1e-2 * plain[far].max() / plain.max()
    c.close()


def test_set_pfb_validation(cuda_ok):
    from paper_1305_5639_gb300._lib import CorrError, CORR_EINVAL

    c = api.Correlator(2, 1, 64, 8)
    w = np.ones((65, 64), np.float32)
    with pytest.raises(CorrError) as e:
        c.set_pfb(w)
    assert e.value.status == CORR_EINVAL
    w = np.ones((2, 64), np.float32)
    w[1, 5] = np.inf
    with pytest.raises(CorrError) as e:
        c.set_pfb(w)
    assert e.value.status == CORR_EINVAL
    c.close()
