"""The tensor-core F-engine (N = 1024 as 32 x 32; both 32-point DFT stages of Eq. 1 as
FP16 hi/lo GEMMs with FP32 accumulation) against the oracle's direct DFT and FP32
re-packing decision.

A code is unique when the oracle's scaled value lies farther than the FP32 error
from a rounding boundary (k + 1/2); those must match bit for bit, the rest may
differ by one. Covered: both output layouts, int8 -128, ragged spectrum counts (a
last item of fewer than 16 spectra, counts that are not multiples of 8), many work
items per persistent CTA, and the
CUDA-core F-engine selected by flag on the same data. The host pipeline's input
blocks (F-engine launches on sub-ranges of the inputs) are covered at N = 1024 in
test_gpu_fx_host_oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"
N = 1024


def _codes(P, planar):
    P = P.cpu().numpy()
    return np.transpose(P, (0, 2, 3, 1)).astype(np.int8) if planar else P


def _check(out, S, scale, bins=None):
    """Unique codes equal, the others within one; returns the fraction unique."""
    sc = scale if bins is None else scale[bins]
    q, margin = oracle.requant(S, sc)
    rms = np.sqrt(np.mean(np.abs(S) ** 2))
    eps = 8 * np.log2(N) * 2.0 ** -24 * rms * sc.max() * 8
    sure = margin > eps
    assert sure.mean() > 0.9
    assert np.array_equal(out[sure], q[sure])
    assert np.all(np.abs(out.astype(np.int32) - q.astype(np.int32)) <= 1)
    assert out.min() >= -127
    return sure.mean()


def _scale(sigma, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.8, 1.25, N) * 16.0 / (sigma * np.sqrt(N))).astype(np.float32)


@pytest.mark.parametrize("planar", [True, False])
@pytest.mark.parametrize("n_ant,n_pol,K", [(3, 1, 40), (1, 2, 16), (2, 1, 8), (1, 1, 37)])
def test_tc_fengine_matches_oracle(cuda_ok, planar, n_ant, n_pol, K):
    if planar and K % 8:
        pytest.skip("the planar layout needs n_spectra % 8 == 0")
    sigma = 48.0
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=K + n_ant, sigma=sigma, lo=-128)
    v[0, :N, 1] = -128  # one frame's imaginary parts all -128
    assert (v == -128).any()
    scale = _scale(sigma, K)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=planar)
    out = _codes(c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)), planar)
    c.check_status()
    _check(out, oracle.channelise(v, N), scale)
    c.close()


def test_tc_fengine_many_items_sampled_bins(cuda_ok):
    """20 inputs x 1000 spectra: 1260 work items, several per CTA, the last item of
    each input ragged (1000 = 62 x 16 + 8); all spectra of a sample of channels."""
    n_ant, n_pol, K = 10, 2, 1000
    bins = [0, 1, 31, 32, 33, 255, 511, 512, 513, 700, 992, 1023]
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=7)
    scale = _scale(16.0, 7)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    P = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV))
    c.check_status()
    out = _codes(P[bins], True)
    del P
    _check(out, oracle.channelise(v, N, bins=bins), scale, bins)
    c.close()


def test_tc_fengine_agrees_with_cudacore_fengine(cuda_ok):
    """The flag-selected CUDA-core F-engine on the same data: both match the oracle's
    unique codes, so they agree there; elsewhere they differ by at most one."""
    n_ant, n_pol, K = 2, 2, 48
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=11)
    scale = _scale(16.0, 11)
    outs = []
    for eng in ("auto", "cudacore"):
        c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True, fengine=eng)
        outs.append(_codes(c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)), True))
        c.check_status()
        c.close()
    S = oracle.channelise(v, N)
    for o in outs:
        _check(o, S, scale)
    assert np.all(np.abs(outs[0].astype(np.int32) - outs[1].astype(np.int32)) <= 1)
    assert (outs[0] != outs[1]).mean() < 1e-3
