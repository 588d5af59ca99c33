"""corr_fx_host end to end against the oracle chain: Eq. 1 (direct DFT), the 8-bit
re-packing (FP32 decision), Eq. 2 in int64 and the FP64 long integration.

The F-engine's FP32 FFT and the oracle's FP64 DFT may round a code differently
when x * scale lies within the FP32 error of a rounding boundary (k + 1/2). Such a
code is 'uncertain' (the oracle's margin says which) and may differ by one; every
visibility no uncertain code enters must equal the oracle's bit for bit, and the
others may differ by no more than the change one-step code flips can make."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _flip_bound(q, unsure):
    """Per (channel, baseline): the largest change of Re or Im of Eq. 2's sum that
    changing each uncertain code component by one can make. q [n_chan, n_in, K, 2]
    int8, unsure [n_chan, n_in, K, 2] bool. A term x_i conj(x_j) moves by at most
    U_i a_j + U_j a_i, with U the number of uncertain components of a sample and a
    = |Re| + |Im| + 2 bounding the (possibly changed) other factor."""
    U = unsure.sum(axis=-1).astype(np.int64)  # [n_chan, n_in, K]
    a = np.abs(q.astype(np.int64)).sum(axis=-1) + 2
    n_in = q.shape[1]
    i, j = oracle.tri_pairs(n_in)
    t = np.einsum("cik,cjk->cij", U, a)  # sum_k U_i a_j
    full = t + np.transpose(t, (0, 2, 1))
    return full[:, i, j]


# 8 inputs (one per copy block), 5 and 9 (fewer inputs than blocks: empty last blocks),
# 12 at N = 1024 (the tensor-core F-engine on sub-ranges of the inputs)
@pytest.mark.parametrize("n_ant,n_pol,N,K", [(4, 2, 64, 64), (5, 1, 256, 24), (3, 3, 64, 32), (6, 2, 1024, 16)])
def test_fx_host_matches_oracle_chain(cuda_ok, n_ant, n_pol, N, K):
    n_in = n_ant * n_pol
    sigma = 16.0
    rng = np.random.default_rng(N + K)  # off powers of two: few exact ties
    scale = (rng.uniform(0.8, 1.25, N) * 16.0 / (sigma * np.sqrt(N))).astype(np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    out = torch.zeros((N, c.n_base), dtype=torch.complex128).pin_memory()
    want = np.zeros((N, c.n_base, 2), np.int64)
    slack = np.zeros((N, c.n_base), np.int64)
    n_exact = 0
    for t in range(2):  # two integrations: the second call adds to the first's FP64 sums
        v = synth.volt_int8(n_ant, n_pol, N, K, seed=300 + 7 * t + N)
        S = oracle.channelise(v, N)  # [N, n_in, K] complex128, Eq. 1
        q, margin = oracle.requant(S, scale)
        eps = 8 * np.log2(N) * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 8
        unsure = margin <= eps
        assert unsure.mean() < 0.01
        want += oracle.cmac(q)  # Eq. 2 in int64, summed as the long integration
        slack += _flip_bound(q, unsure)
        c.fx_host(torch.from_numpy(v).pin_memory(), torch.from_numpy(scale).to(DEV), out)
        torch.cuda.synchronize()
        got = out.numpy()
        dre = np.abs(got.real - want[..., 0])
        dim = np.abs(got.imag - want[..., 1])
        sure = slack == 0
        assert np.array_equal(got.real[sure], want[..., 0][sure].astype(np.float64)), t
        assert np.array_equal(got.imag[sure], want[..., 1][sure].astype(np.float64)), t
        assert np.all(dre <= slack) and np.all(dim <= slack), t
        n_exact = sure.mean()
    assert n_exact > 0.5  # most visibilities are pinned exactly
    c.check_status()
    c.close()


@pytest.mark.parametrize("n_ant,n_pol,N,K", [(4, 2, 64, 64), (6, 2, 1024, 16)])
def test_fx_host_accum_matches_oracle_chain(cuda_ok, n_ant, n_pol, N, K):
    """corr_fx_host_accum: each call's INT32 output is that integration alone (oracle
    chain, same bound for codes near a rounding tie), and the FP64 long integration it
    keeps on the device is the exact sum of the calls' outputs."""
    n_in = n_ant * n_pol
    sigma = 16.0
    rng = np.random.default_rng(N + K + 1)
    scale = (rng.uniform(0.8, 1.25, N) * 16.0 / (sigma * np.sqrt(N))).astype(np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    acc = torch.zeros((N, c.n_base, 2), dtype=torch.int32).pin_memory()
    total = np.zeros((N, c.n_base, 2), np.int64)
    for t in range(2):
        v = synth.volt_int8(n_ant, n_pol, N, K, seed=500 + 3 * t + N, lo=-128)
        S = oracle.channelise(v, N)
        q, margin = oracle.requant(S, scale)
        eps = 8 * np.log2(N) * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 8
        unsure = margin <= eps
        want = oracle.cmac(q)
        slack = _flip_bound(q, unsure)
        c.fx_host_accum(torch.from_numpy(v).pin_memory(), torch.from_numpy(scale).to(DEV), acc)
        torch.cuda.synchronize()
        got = acc.numpy().astype(np.int64)
        sure = slack == 0
        assert sure.mean() > 0.5
        for comp in range(2):
            assert np.array_equal(got[..., comp][sure], want[..., comp][sure]), t
            assert np.all(np.abs(got[..., comp] - want[..., comp]) <= slack), t
        total += got
    vis = c.dump().cpu().numpy()  # the FP64 long integration of both calls
    assert np.array_equal(vis.real, total[..., 0].astype(np.float64))
    assert np.array_equal(vis.imag, total[..., 1].astype(np.float64))
    c.check_status()
    c.close()


def test_fx_host_accum_rejections(cuda_ok):
    """No INT32 accumulator with the fused dump; NULL buffers are rejected."""
    n_ant, n_pol, N, K = 2, 2, 64, 16
    v = torch.from_numpy(synth.volt_int8(n_ant, n_pol, N, K, seed=9)).pin_memory()
    scale = torch.full((N,), 0.125, device=DEV)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True, fused_dump=True)
    acc = torch.zeros((N, c.n_base, 2), dtype=torch.int32).pin_memory()
    with pytest.raises(api.CorrError) as e:
        c.fx_host_accum(v, scale, acc)
    assert e.value.status == api._lib.CORR_EUNSUPPORTED
    c.close()
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    st = api._lib.load().corr_fx_host_accum(c.h, None, api._ptr(scale), api._hptr(acc), None)
    assert st == api._lib.CORR_EINVAL
    st = api._lib.load().corr_fx_host_accum(c.h, api._hptr(v), api._ptr(scale), None, None)
    assert st == api._lib.CORR_EINVAL
    c.close()
