"""Parity of the CUDA path (through the C ABI) with the FP64 oracle: F-engine,
CUDA-core X-engines, gains, dump, adjoint. Seeded synthetic inputs from synth;
sizes span several tiles plus ragged tails."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api
from paper_1305_5639_gb300._lib import CorrError, CORR_EOVERFLOW, CORR_EINVAL

pytestmark = pytest.mark.gpu

DEV = "cuda"


def norm_err(V, Vref, n_in):
    """e_ij = |V_ij - Vref_ij| / sqrt(|Vref_ii| |Vref_jj|); returns (max, rms)."""
    i, j = oracle.tri_pairs(n_in)
    d = np.abs(V - Vref)
    aut = np.abs(Vref[..., oracle.packed_index(np.arange(n_in), np.arange(n_in))])
    den = np.sqrt(aut[..., i] * aut[..., j])
    e = d / den
    return float(np.max(e)), float(np.sqrt(np.mean(e ** 2)))


def c64(V2):
    """[..., 2] float -> complex128."""
    return V2[..., 0].astype(np.float64) + 1j * V2[..., 1].astype(np.float64)


# --------------------------------------------------------------------------- F-engine
@pytest.mark.parametrize("N,n_in,K", [(16, 3, 21), (64, 2, 9), (128, 3, 10), (256, 3, 13), (512, 2, 7),
                                     (1024, 2, 11), (2048, 2, 5), (4096, 2, 3)])
def test_fengine_fp32_matches_dft(cuda_ok, N, n_in, K):
    v = synth.volt_fp32(n_in, N, K, seed=N)
    c = api.Correlator(n_in, 1, N, K, precision="fp32")
    S = c.fengine(torch.from_numpy(v).to(DEV)).cpu().numpy().astype(np.complex128)
    ref = oracle.channelise(v, N)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(S - ref)) <= 1e-5 * rms
    c.close()


@pytest.mark.parametrize("N,n_ant,n_pol,K", [(16, 2, 2, 37), (64, 3, 1, 20), (128, 2, 2, 19), (256, 2, 2, 17),
                                            (512, 1, 2, 21), (1024, 1, 2, 35), (2048, 1, 2, 13), (4096, 1, 2, 9)])
def test_fengine_int8_requant_corner_turn(cuda_ok, N, n_ant, n_pol, K):
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=7)
    rng = np.random.default_rng(N)
    scale = (rng.uniform(0.8, 1.25, N) / np.sqrt(N)).astype(np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8")
    q_gpu = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    S = oracle.channelise(v, N)
    q, margin = oracle.requant(S, scale)
    # codes decided more than the FP32 FFT error away from a .5 boundary are unique
    eps = 8 * np.log2(N) * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 4
    sure = margin > eps
    assert np.array_equal(q_gpu[sure], q[sure])
    assert np.all(np.abs(q_gpu.astype(np.int32) - q.astype(np.int32)) <= 1)
    assert q_gpu.min() >= -127
    c.close()


def test_fengine_unaligned_input_rejected(cuda_ok):
    """Raw voltages must start on a 16-byte boundary (the F-engine copies whole
    frames asynchronously in 16-byte pieces): an offset view is refused."""
    N, K = 1024, 8
    v = torch.zeros((2, K * N, 2), dtype=torch.int8, device=DEV)
    raw = torch.empty(v.numel() + 16, dtype=torch.uint8, device=DEV)
    vu = raw[2:2 + v.numel()].view(torch.int8).view(v.shape)
    c = api.Correlator(2, 1, N, K, precision="int8", planar=True)
    sc = torch.ones(N, device=DEV)
    for call in (lambda: c.fengine(vu, sc), lambda: c.fengine_power(vu)):
        with pytest.raises(CorrError) as e:
            call()
        assert e.value.status == CORR_EINVAL
    c.close()


def test_fengine_power(cuda_ok):
    n_in, N, K = 4, 256, 24
    v = synth.volt_fp32(n_in, N, K, seed=5)
    c = api.Correlator(n_in, 1, N, K)
    p = c.fengine_power(torch.from_numpy(v).to(DEV)).cpu().numpy()
    ref = oracle.channel_power(oracle.channelise(v, N))
    assert np.allclose(p, ref, rtol=1e-4)
    c.close()


# --------------------------------------------------------------------------- X-engine (CUDA cores)
# few inputs (<= 22: one CTA per channel, one thread per pair) and the tiled kernel
@pytest.mark.parametrize("n_in,K,n_chan", [(70, 37, 3), (16, 64, 2), (1, 5, 2), (129, 16, 1), (22, 131, 3),
                                         (23, 40, 2), (8, 1000, 2)])
def test_xengine_cudacore_fp32(cuda_ok, n_in, K, n_chan):
    X = synth.chan_sources(n_chan, n_in, K, n_src=2, seed=1, src_amp=0.5)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp32", xengine="cudacore")
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    ref = oracle.cmac(X)
    emax, _ = norm_err(V, ref, n_in)
    assert emax <= 1e-5
    c.close()


@pytest.mark.parametrize("n_in,K,n_chan", [(70, 45, 2), (64, 32, 1), (3, 7, 3), (130, 64, 1)])
def test_xengine_cudacore_int8_exact(cuda_ok, n_in, K, n_chan):
    X = synth.chan_int8(n_chan, n_in, K, seed=2)
    X[0, 0] = 127
    if n_in > 1:
        X[0, 1] = -127
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", xengine="cudacore")
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    assert np.array_equal(V, oracle.cmac(X))
    c.close()


@pytest.mark.parametrize("n_in", [40, 16])
def test_xengine_gains_fp32(cuda_ok, n_in):
    K, n_chan = 24, 2
    X = synth.chan_sources(n_chan, n_in, K, n_src=1, seed=3, src_amp=0.3)
    g = synth.gains(n_in, seed=3)
    c = api.Correlator(n_in, 1, n_chan, K)
    c.xengine(torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    ref = oracle.apply_gains(oracle.cmac(X), g, n_in)
    emax, _ = norm_err(V, ref, n_in)
    assert emax <= 1e-5
    c.close()


@pytest.mark.parametrize("n_in", [40, 16])
def test_xengine_fp32_accumulates_two_calls(cuda_ok, n_in):
    # the second call of an integration adds to the first (both FP32 kernels)
    K, n_chan = 70, 2
    X1 = synth.chan_sources(n_chan, n_in, K, n_src=1, seed=4, src_amp=0.3)
    X2 = synth.chan_sources(n_chan, n_in, K, n_src=1, seed=5, src_amp=0.3)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp32", xengine="cudacore")
    c.xengine(torch.from_numpy(X1).to(DEV))
    c.xengine(torch.from_numpy(X2).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    ref = oracle.cmac(np.concatenate([X1, X2], axis=2))
    emax, _ = norm_err(V, ref, n_in)
    assert emax <= 1e-5
    c.close()


def test_gains_rejected_for_int8(cuda_ok):
    c = api.Correlator(4, 1, 2, 8, precision="int8")
    X = torch.zeros((2, 4, 8, 2), dtype=torch.int8, device=DEV)
    g = torch.ones(4, dtype=torch.complex64, device=DEV)
    with pytest.raises(CorrError) as e:
        c.xengine(X, g)
    assert e.value.status == CORR_EINVAL
    c.close()


def test_dump_accumulates_integrations_fp64(cuda_ok):
    n_in, K, n_chan = 33, 16, 2
    parts = [synth.chan_int8(n_chan, n_in, K, seed=10 + p) for p in range(3)]
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", xengine="cudacore")
    c.xengine(torch.from_numpy(parts[0]).to(DEV))
    c.xengine(torch.from_numpy(parts[1]).to(DEV))  # two integrations in the accumulator
    c.dump(copy=False)
    c.xengine(torch.from_numpy(parts[2]).to(DEV))
    vis = c.dump().cpu().numpy()
    want = oracle.dump([oracle.cmac(p) for p in parts])
    assert np.array_equal(vis, want[..., 0] + 1j * want[..., 1])
    assert np.all(c.accum().cpu().numpy() == 0)  # dump clears the accumulator
    c.close()


def test_int8_overflow_guard_across_calls(cuda_ok):
    K = 40000
    c = api.Correlator(2, 1, 1, K, precision="int8", xengine="cudacore")
    X = torch.zeros((1, 2, K, 2), dtype=torch.int8, device=DEV)
    c.xengine(X)
    with pytest.raises(CorrError) as e:
        c.xengine(X)
    assert e.value.status == CORR_EOVERFLOW
    c.dump(copy=False)
    c.xengine(X)  # allowed again after the dump
    c.close()


# --------------------------------------------------------------------------- full FX, config A
def test_config_A_full_fx_fp32(cuda_ok):
    cfg = synth.CONFIGS["A"]
    n_in, N, K = cfg["n_ant"] * cfg["n_pol"], cfg["n_chan"], cfg["n_spectra"]
    v = synth.volt_fp32(n_in, N, K, seed=0)
    c = api.Correlator(cfg["n_ant"], cfg["n_pol"], N, K, precision="fp32")
    chan = c.fengine(torch.from_numpy(v).to(DEV))
    c.xengine(chan)
    vis = c.dump().cpu().numpy()
    ref = oracle.cmac(oracle.channelise(v, N))
    emax, erms = norm_err(vis, ref, n_in)
    assert emax <= 1e-5, (emax, erms)
    # the delayed source's lag peak is where the oracle puts it
    i, j = oracle.tri_pairs(n_in)
    peak = np.argmax(np.abs(np.fft.ifft(vis, axis=0)), axis=0)
    assert np.array_equal(peak[i != j], ((i - j) % N)[i != j])
    c.close()


# --------------------------------------------------------------------------- adjoint
def _calib_case(n_chan, n_in, K, seed, auto_w=0.0):
    X = synth.chan_sources(n_chan, n_in, K, n_src=5, seed=seed)
    g = synth.gains(n_in, seed=seed)
    M = synth.sky_model(n_chan, n_in, 5, seed=seed)
    w = synth.weights(n_in, auto_w)
    return X, g, M, w


@pytest.mark.parametrize("n_in,K,n_chan,auto_w", [(70, 80, 3, 0.0), (33, 17, 2, 1.0)])
def test_backward_matches_oracle_gradient(cuda_ok, n_in, K, n_chan, auto_w):
    X, g, M, w = _calib_case(n_chan, n_in, K, seed=4, auto_w=auto_w)
    L, dX_ref, dg_ref = oracle.loss_and_grads(X, g, M, w)
    Vp = oracle.apply_gains(oracle.cmac(X), g, n_in)
    G = (2.0 * w * (Vp / K - M) / K).astype(np.complex64)  # dL/dV' (oracle side)
    c = api.Correlator(n_in, 1, n_chan, K)
    dX, dg = c.backward(torch.from_numpy(G).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
    dX = dX.cpu().numpy()
    dg = dg.cpu().numpy()
    assert np.linalg.norm(dX - dX_ref) <= 1e-4 * np.linalg.norm(dX_ref)
    assert np.linalg.norm(dg - dg_ref) <= 1e-4 * np.linalg.norm(dg_ref)
    # element-wise, per channel: max error over the channel's rms (10x the L2 bar)
    rms = np.sqrt(np.mean(np.abs(dX_ref) ** 2, axis=(1, 2)))
    assert np.max(np.max(np.abs(dX - dX_ref), axis=(1, 2)) / rms) <= 1e-3
    assert np.max(np.abs(dg - dg_ref)) <= 1e-3 * np.sqrt(np.mean(np.abs(dg_ref) ** 2))
    c.close()


def test_autograd_corrfn_end_to_end(cuda_ok):
    from paper_1305_5639_gb300.autograd import CorrFn

    n_in, K, n_chan = 24, 32, 2
    X, g, M, w = _calib_case(n_chan, n_in, K, seed=6)
    L_ref, dX_ref, dg_ref = oracle.loss_and_grads(X, g, M, w)
    c = api.Correlator(n_in, 1, n_chan, K)
    Xt = torch.from_numpy(X).to(DEV).requires_grad_(True)
    gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
    Mt = torch.from_numpy(M).to(DEV)
    wt = torch.from_numpy(w).to(DEV)
    V = CorrFn.apply(Xt, gt, c)
    R = V.to(torch.complex128) / K - Mt
    L = torch.sum(wt * (R.real ** 2 + R.imag ** 2))
    L.backward()
    assert abs(L.item() - L_ref) <= 1e-4 * abs(L_ref)
    assert np.linalg.norm(gt.grad.cpu().numpy() - dg_ref) <= 1e-4 * np.linalg.norm(dg_ref)
    assert np.linalg.norm(Xt.grad.cpu().numpy() - dX_ref) <= 1e-4 * np.linalg.norm(dX_ref)
    c.close()
