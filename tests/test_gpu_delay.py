"""Delay compensation fused into the F-engine against the oracle's delay-compensated
channelisation (integer advance, Eq. 1, fractional phase per channel)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _delays(n_in, N, seed):
    """Mixed delays: zero, fractional, negative, beyond one frame, a half."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-1.5 * N, 1.5 * N, n_in).astype(np.float32)
    d[0] = 0.0
    if n_in > 1:
        d[1] = 2.5
    if n_in > 2:
        d[2] = -0.25
    return d


@pytest.mark.parametrize("N,n_in,K", [(16, 5, 21), (64, 3, 9), (128, 3, 8), (256, 3, 13), (512, 2, 9),
                                     (1024, 4, 11), (2048, 2, 5), (4096, 2, 4)])
def test_fengine_fp32_delays_match_oracle(cuda_ok, N, n_in, K):
    v = synth.volt_fp32(n_in, N, K, seed=N + 1)
    d = _delays(n_in, N, seed=N)
    c = api.Correlator(n_in, 1, N, K, precision="fp32")
    c.set_delays(d)
    S = c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy().astype(np.complex128)
    ref = oracle.channelise_delayed(v, N, d)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(S - ref)) <= 1e-5 * rms
    # switching compensation off gives the plain channeliser's result again
    c.set_delays(None)
    S0 = c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(S0 - oracle.channelise(v, N))) <= 1e-5 * rms
    c.close()


@pytest.mark.parametrize("planar", [False, True])
@pytest.mark.parametrize("N,n_ant,n_pol,K", [(64, 3, 1, 24), (256, 2, 2, 16), (512, 1, 2, 16), (1024, 1, 2, 40),
                                            (4096, 1, 2, 8)])
def test_fengine_int8_delays_requant(cuda_ok, planar, N, n_ant, n_pol, K):
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=9)
    n_in = n_ant * n_pol
    d = _delays(n_in, N, seed=N + 7)
    rng = np.random.default_rng(N)
    scale = (rng.uniform(0.8, 1.25, N) / np.sqrt(N)).astype(np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=planar)
    c.set_delays(d)
    out = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    if planar:  # [N][2][n_in][K] FP16 codes -> [N][n_in][K][2]
        out = np.transpose(out, (0, 2, 3, 1)).astype(np.int8)
    S = oracle.channelise_delayed(v, N, d)
    q, margin = oracle.requant(S, scale)
    eps = 8 * np.log2(N) * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 8
    sure = margin > eps
    assert np.array_equal(out[sure], q[sure])
    assert np.all(np.abs(out.astype(np.int32) - q.astype(np.int32)) <= 1)
    c.close()


def test_fengine_delays_tone_has_zero_phase(cuda_ok):
    """A tone at bin k0 delayed by tau_i comes out of the compensated F-engine with
    zero phase in every frame whose advanced samples are recorded."""
    N, K, k0 = 256, 8, 37
    tau = np.array([0.0, 3.3, -2.7, 300.6], np.float32)
    t = np.arange(K * N)
    v = np.exp(2j * np.pi * k0 * (t[None, :] - tau.astype(np.float64)[:, None]) / N).astype(np.complex64)
    c = api.Correlator(len(tau), 1, N, K, precision="fp32")
    c.set_delays(tau)
    S = c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy()
    D, _ = oracle.delay_split(tau)
    for i in range(len(tau)):
        a_lo = int(np.ceil(max(0, -D[i]) / N))
        a_hi = K - int(np.ceil(max(0, D[i]) / N))
        z = S[k0, i, a_lo:a_hi]
        assert np.allclose(np.abs(z), N, rtol=1e-5), i
        assert np.max(np.abs(np.angle(z))) <= 2e-5, i
    c.close()


def test_power_pass_with_delays(cuda_ok):
    n_in, N, K = 3, 64, 20
    v = synth.volt_fp32(n_in, N, K, seed=13)
    d = np.array([0.0, 17.4, -40.5], np.float32)
    c = api.Correlator(n_in, 1, N, K)
    c.set_delays(d)
    p = c.fengine_power(torch.from_numpy(v).to(DEV)).cpu().numpy()
    ref = oracle.channel_power(oracle.channelise_delayed(v, N, d))
    assert np.allclose(p, ref, rtol=1e-4)
    c.close()


def test_delay_compensation_aligns_cross_phases(cuda_ok):
    """One broadband stream reaching the inputs with whole-sample delays d_i: without
    compensation the cross-correlation phases follow the ramp -2 pi k (d_i - d_j) / N;
    with it they vanish (up to the frames cut by the record's end)."""
    n_in, N, K = 6, 64, 256
    d = np.array([0, 3, 7, 12, 30, 45])
    v = synth.volt_fp32(n_in, N, K, seed=3, src_amp=1.0, delays=d, noise=False)
    c = api.Correlator(n_in, 1, N, K, precision="fp32", xengine="cudacore")
    ii, jj = oracle.tri_pairs(n_in)
    cross = ii != jj
    for comp in (False, True):
        c.set_delays(d.astype(np.float32) if comp else None)
        c.reset()
        c.xengine(c.fengine(torch.from_numpy(v).to(DEV)))
        V = c.accum().cpu().numpy()[:, cross]
        ph = np.abs(np.angle(V))
        if comp:
            assert np.median(ph) < 0.02
        else:
            assert np.median(ph) > 0.5
    c.close()


def test_set_delays_validation(cuda_ok):
    from paper_1305_5639_gb300._lib import CorrError, CORR_EINVAL, CORR_EUNSUPPORTED

    c = api.Correlator(4, 1, 64, 8)
    with pytest.raises(CorrError) as e:
        c.set_delays(np.array([0, np.nan, 0, 0], np.float32))
    assert e.value.status == CORR_EINVAL
    with pytest.raises(CorrError) as e:
        c.set_delays(np.array([0, 2e9, 0, 0], np.float32))
    assert e.value.status == CORR_EINVAL
    c.close()
    c = api.Correlator(4, 1, 48, 8)  # 48 channels: no F-engine
    with pytest.raises(CorrError) as e:
        c.set_delays(np.zeros(4, np.float32))
    assert e.value.status == CORR_EUNSUPPORTED
    c.close()
