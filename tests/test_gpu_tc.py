"""Parity of the tcgen05 tensor-core X-engine (through the C ABI) with the FP64
oracle: INT8 bit-exact, FP16 within its stated tolerance; ragged sizes span
several tiles, several 512-spectrum INT32 folds and partial pipeline stages."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def norm_err(V, Vref, n_in):
    i, j = oracle.tri_pairs(n_in)
    aut = np.abs(Vref[..., oracle.packed_index(np.arange(n_in), np.arange(n_in))])
    e = np.abs(V - Vref) / np.sqrt(aut[..., i] * aut[..., j])
    return float(np.max(e)), float(np.sqrt(np.mean(e ** 2)))


@pytest.mark.parametrize("n_in,K,n_chan", [
    (128, 64, 1),      # one diagonal tile, one stage
    (256, 640, 2),     # 3 tiles, two INT32 folds (512 + 128 spectra)
    (200, 100, 3),     # ragged inputs, K not a multiple of 8 (scalar loads)
    (130, 1032, 1),    # 2 x 2 blocks with a 2-input tail, 3 folds, partial last stage
    (1, 8, 2),         # a single input
    (384, 136, 1),     # 6 tiles
])
def test_tc_int8_bit_exact(cuda_ok, n_in, K, n_chan):
    X = synth.chan_int8(n_chan, n_in, K, seed=n_in + K)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", xengine="tcgen05")
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    assert np.array_equal(V, oracle.cmac(X))
    c.close()


def test_tc_int8_extreme_values_exact(cuda_ok):
    """All samples at +-127 for 4096 spectra: autos reach 2 * 127^2 * 4096, far
    beyond 2^24, and each 512-spectrum FP32 partial reaches its bound."""
    n_in, K = 160, 4096
    X = np.empty((1, n_in, K, 2), np.int8)
    rng = np.random.default_rng(0)
    X[...] = np.where(rng.random((1, n_in, K, 2)) < 0.5, 127, -127)
    X[0, :8] = 127
    X[0, 8:16] = -127
    c = api.Correlator(n_in, 1, 1, K, precision="int8", xengine="tcgen05")
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    assert np.array_equal(V, oracle.cmac(X))
    c.close()


def test_tc_int8_equals_cudacore_and_accumulates(cuda_ok):
    n_in, K, n_chan = 300, 520, 4
    X1 = synth.chan_int8(n_chan, n_in, K, seed=1)
    X2 = synth.chan_int8(n_chan, n_in, K, seed=2)
    out = []
    for eng in ("tcgen05", "cudacore"):
        c = api.Correlator(n_in, 1, n_chan, K, precision="int8", xengine=eng)
        c.xengine(torch.from_numpy(X1).to(DEV))
        c.xengine(torch.from_numpy(X2).to(DEV))  # second call adds into the accumulator
        out.append(c.accum().cpu().numpy())
        c.close()
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[0].astype(np.int64), oracle.cmac(X1) + oracle.cmac(X2))


def test_tc_int8_deterministic(cuda_ok):
    n_in, K = 256, 256
    X = torch.from_numpy(synth.chan_int8(2, n_in, K, seed=5)).to(DEV)
    c = api.Correlator(n_in, 1, 2, K, precision="int8")
    c.xengine(X)
    a = c.accum()
    c.reset()
    c.xengine(X)
    b = c.accum()
    assert torch.equal(a, b)
    c.close()


@pytest.mark.parametrize("n_in,K,n_chan", [(128, 256, 2), (250, 200, 2), (70, 33, 1)])
def test_tc_fp16_plain(cuda_ok, n_in, K, n_chan):
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=3, src_amp=0.1)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16")
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    emax, erms = norm_err(V, oracle.cmac(X), n_in)
    assert emax <= 2e-3, (emax, erms)
    c.close()


def test_tc_fp16_gains(cuda_ok):
    n_in, K, n_chan = 140, 128, 2
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=8, src_amp=0.1)
    g = synth.gains(n_in, seed=8)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16")
    c.xengine(torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    ref = oracle.apply_gains(oracle.cmac(X), g, n_in)
    emax, _ = norm_err(V, ref, n_in)
    assert emax <= 2e-3
    c.close()


# --------------------------------------------------------------------------- planar FP16 layout + TMA X-engine
def to_planar(X):
    """complex int8 [n_chan, n_in, K, 2] -> planar FP16 [n_chan, 2, n_in, K] (same integer values)."""
    return np.ascontiguousarray(np.transpose(X, (0, 3, 1, 2)).astype(np.float16))


@pytest.mark.parametrize("n_in,K,n_chan", [
    (128, 64, 1),      # one diagonal tile, one stage
    (256, 640, 2),     # 3 tiles, two 512-spectrum folds on alternating accumulators
    (200, 104, 3),     # ragged inputs and a partial stage (TMA zero fill)
    (130, 1032, 1),    # 2 x 2 blocks, 3 folds
    (1, 8, 2),         # a single input
    (512, 4096, 2),    # the INT8 workload's channel shape
])
def test_tma_planar_int8_bit_exact(cuda_ok, n_in, K, n_chan):
    X = synth.chan_int8(n_chan, n_in, K, seed=n_in + 7 * K)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    c.xengine(torch.from_numpy(to_planar(X)).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    assert np.array_equal(V, oracle.cmac(X))
    c.close()


def test_tma_planar_extreme_values_and_accumulate(cuda_ok):
    n_in, K = 160, 4096
    rng = np.random.default_rng(1)
    X = np.where(rng.random((1, n_in, K, 2)) < 0.5, 127, -127).astype(np.int8)
    X[0, :8] = 127
    c = api.Correlator(n_in, 1, 1, K, precision="int8", planar=True)
    P = torch.from_numpy(to_planar(X)).to(DEV)
    c.xengine(P)
    c.xengine(P)  # accumulate a second integration (INT32 guard allows 2 x 4096)
    V = c.accum().cpu().numpy().astype(np.int64)
    assert np.array_equal(V, 2 * oracle.cmac(X))
    c.close()


@pytest.mark.parametrize("N", [128, 512, 1024, 2048, 4096])
def test_fengine_planar_matches_int8_layout_and_oracle(cuda_ok, N):
    n_ant, n_pol, K = 3, 2, 40
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=9)
    scale = np.full(N, 0.5 / np.sqrt(N), np.float32)  # rms 16 sqrt(N) -> 8
    vt, st = torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)
    a = api.Correlator(n_ant, n_pol, N, K, precision="int8")
    b = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    q8 = a.fengine(vt, st).cpu().numpy()            # [N, n_in, K, 2] int8
    qp = b.fengine(vt, st).cpu().numpy()            # [N, 2, n_in, K] float16
    assert np.array_equal(to_planar(q8), qp)
    S = oracle.channelise(v, N)
    q, margin = oracle.requant(S, scale)
    sure = margin > 1e-3
    assert np.array_equal(q8[sure], q[sure])
    a.close()
    b.close()


def test_full_fx_planar_int8_workload_shape(cuda_ok):
    """F-engine -> planar -> TMA X-engine on a channel subset of the INT8 workload's
    shape, against the oracle's own chain (direct DFT, FP32 re-packing decision,
    int64 CMAC). Codes may differ only next to a rounding boundary, and by one; on
    every channel whose codes all agree the visibilities must be identical."""
    n_ant, n_pol, N, K = 16, 2, 1024, 256
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=11)
    scale = np.full(N, 1.0 / 32.0, np.float32)  # rms 16 sqrt(N) -> 16
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    P = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV))
    c.xengine(P)
    V = c.accum().cpu().numpy().astype(np.int64)
    sel = [0, 1, 5, 100, 511, 512, 777, 1023]
    S = oracle.channelise(v, N, bins=sel)
    q, margin = oracle.requant(S, scale[sel])
    Vref = oracle.cmac(q)
    q_gpu = np.transpose(P.cpu().numpy()[sel], (0, 2, 3, 1)).astype(np.int8)  # compared, not fed to the oracle
    diff = q_gpu != q
    assert np.all(margin[diff] < 1e-3)
    assert np.all(np.abs(q_gpu[diff].astype(int) - q[diff].astype(int)) == 1)
    checked = 0
    for t, k in enumerate(sel):
        if not diff[t].any():
            assert np.array_equal(V[k], Vref[t]), k
            checked += 1
    assert checked >= 4
    c.close()


def test_tma_fused_dump_equals_separate_dump(cuda_ok):
    """The FP64 long integration fed straight from the X-engine epilogue equals the
    oracle's sum of integrations (exact: integer sums below 2^53)."""
    from paper_1305_5639_gb300._lib import CorrError, CORR_ESTATE

    n_in, K, n_chan = 300, 1024, 2
    parts = [synth.chan_int8(n_chan, n_in, K, seed=40 + t) for t in range(3)]
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True, fused_dump=True)
    for X in parts:
        c.xengine(torch.from_numpy(to_planar(X)).to(DEV))
    vis = c.dump().cpu().numpy()
    want = oracle.dump([oracle.cmac(X) for X in parts])
    assert np.array_equal(vis, want[..., 0] + 1j * want[..., 1])
    with pytest.raises(CorrError) as e:
        c.accum()
    assert e.value.status == CORR_ESTATE
    for _ in range(20):  # many integrations: no INT32 guard applies across calls
        c.xengine(torch.from_numpy(to_planar(parts[0])).to(DEV))
    c.check_status()
    c.close()


# --------------------------------------------------------------------------- FP16 hi/lo and plain on the TMA path
@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("fp16_hilo", 5e-5)])
@pytest.mark.parametrize("n_in,K,n_chan", [(128, 256, 2), (250, 200, 2), (300, 520, 1)])
def test_tma_fp16_paths(cuda_ok, prec, tol, n_in, K, n_chan):
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=n_in, src_amp=0.1)
    c = api.Correlator(n_in, 1, n_chan, K, precision=prec)
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    c.check_status()
    emax, erms = norm_err(V, oracle.cmac(X), n_in)
    assert emax <= tol, (emax, erms)
    c.close()


def test_tma_fp16_hilo_gains_and_explicit_tcgen05(cuda_ok):
    n_in, K, n_chan = 140, 128, 2
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=8, src_amp=0.1)
    g = synth.gains(n_in, seed=8)
    ref = oracle.apply_gains(oracle.cmac(X), g, n_in)
    for prec, eng, tol in (("fp16_hilo", "auto", 5e-5), ("fp16", "tcgen05", 2e-3)):
        c = api.Correlator(n_in, 1, n_chan, K, precision=prec, xengine=eng)
        c.xengine(torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
        V = c.accum().cpu().numpy().astype(np.complex128)
        emax, _ = norm_err(V, ref, n_in)
        assert emax <= tol, (prec, eng, emax)
        c.close()


@pytest.mark.parametrize("prec", ["fp16", "fp16_hilo"])
@pytest.mark.parametrize("with_gains", [False, True])
def test_tma_fp16_fused_dump_equals_separate_dump(cuda_ok, prec, with_gains):
    """FP16 / hi-lo with the dump fused into the X-engine epilogue: bit-identical to
    the separate dump (the same FP32 tile sums are added in FP64), three integrations."""
    from paper_1305_5639_gb300._lib import CorrError, CORR_ESTATE

    n_in, K, n_chan = 200, 136, 3
    parts = [synth.chan_sources(n_chan, n_in, K, n_src=3, seed=70 + t, src_amp=0.1) for t in range(3)]
    g = torch.from_numpy(synth.gains(n_in, seed=7)).to(DEV) if with_gains else None
    sep = api.Correlator(n_in, 1, n_chan, K, precision=prec)
    fus = api.Correlator(n_in, 1, n_chan, K, precision=prec, fused_dump=True)
    for X in parts:
        Xt = torch.from_numpy(X).to(DEV)
        sep.xengine(Xt, g)
        sep.dump(copy=False)
        fus.xengine(Xt, g)
    a, b = sep.dump().cpu().numpy(), fus.dump().cpu().numpy()
    fus.check_status()
    assert np.array_equal(a, b)
    with pytest.raises(CorrError) as e:
        fus.accum()
    assert e.value.status == CORR_ESTATE
    sep.close()
    fus.close()


def test_fused_dump_flag_validation(cuda_ok):
    """The fused dump lives in the tensor-core X-engine's epilogue: FP32 and the
    CUDA-core X-engines refuse it."""
    from paper_1305_5639_gb300._lib import CorrError, CORR_EUNSUPPORTED

    for kw in (dict(precision="fp32"), dict(precision="int8", xengine="cudacore"),
               dict(precision="fp32", xengine="tcgen05")):
        with pytest.raises(CorrError) as e:
            api.Correlator(16, 1, 2, 64, fused_dump=True, **kw)
        assert e.value.status == CORR_EUNSUPPORTED, kw


@pytest.mark.parametrize("prec,K", [("int8", 100), ("fp16", 60), ("fp16_hilo", 37)])
def test_fused_dump_any_layout_and_ragged_spectra(cuda_ok, prec, K):
    """Complex int8 and complex float inputs (converted to planar operands by the
    library, spectra padded to a multiple of 8) with the dump fused: equal to the
    separate dump over two integrations."""
    n_in, n_chan = 150, 2
    if prec == "int8":
        parts = [synth.chan_int8(n_chan, n_in, K, seed=90 + t) for t in range(2)]
    else:
        parts = [synth.chan_sources(n_chan, n_in, K, n_src=3, seed=90 + t, src_amp=0.1) for t in range(2)]
    sep = api.Correlator(n_in, 1, n_chan, K, precision=prec)
    fus = api.Correlator(n_in, 1, n_chan, K, precision=prec, fused_dump=True)
    for X in parts:
        Xt = torch.from_numpy(X).to(DEV)
        sep.xengine(Xt)
        sep.dump(copy=False)
        fus.xengine(Xt)
    a, b = sep.dump().cpu().numpy(), fus.dump().cpu().numpy()
    fus.check_status()
    assert np.array_equal(a, b)
    if prec == "int8":
        want = oracle.dump([oracle.cmac(X) for X in parts])
        assert np.array_equal(a, want[..., 0] + 1j * want[..., 1])
    sep.close()
    fus.close()


def test_fp16_workload_channel_two_integrations(cuda_ok):
    """The FP16 workload's full channel shape (1024 antennas x 2 pol = 2048 inputs,
    2048 spectra per integration, 3 sources) on one channel, two integrations dumped
    to FP64, plain FP16 and hi/lo, against the oracle."""
    n_in, K = 2048, 2048
    chans = [1234]
    parts = [synth.chan_sources(4096, n_in, K, n_src=3, seed=21 + t, chans=chans, src_amp=0.1) for t in range(2)]
    ref = oracle.dump([oracle.cmac(X) for X in parts])
    for prec, tol in (("fp16", 2e-3), ("fp16_hilo", 5e-5)):
        c = api.Correlator(1024, 2, 1, K, precision=prec)
        for X in parts:
            c.xengine(torch.from_numpy(X).to(DEV))
            c.dump(copy=False)
        vis = c.dump().cpu().numpy()
        emax, erms = norm_err(vis, ref, n_in)
        assert emax <= tol, (prec, emax, erms)
        c.close()


# --------------------------------------------------------------------------- host-buffer pipeline
@pytest.mark.parametrize("fused", [False, True])
def test_fx_host_pipeline_equals_device_path(cuda_ok, fused):
    """corr_fx_host (pinned host voltages in, FP64 visibilities out, copies
    overlapped with the engines block by block) gives exactly the device path's
    result, and a second call adds a second integration."""
    n_ant, n_pol, N, K = 20, 2, 256, 256  # 40 inputs: 8 uneven input blocks
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=31)
    scale = torch.full((N,), 1.0 / 16.0, device=DEV)
    vt = torch.from_numpy(v).to(DEV)
    ref = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    ref.xengine(ref.fengine(vt, scale))
    ref.dump(copy=False)
    want1 = ref.dump().cpu().numpy()
    ref.xengine(ref.fengine(vt, scale))
    want2 = ref.dump().cpu().numpy()
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True, fused_dump=fused)
    vh = torch.from_numpy(v).pin_memory()
    out = torch.zeros((N, c.n_base), dtype=torch.complex128).pin_memory()
    c.fx_host(vh, scale, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), want1)
    c.fx_host(vh, scale, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy(), want2)
    c.check_status()
    c.close()
    ref.close()


def test_fx_host_back_to_back_calls(cuda_ok):
    """Calls issued without synchronising in between (the copy-in of one overlaps
    the previous call's X-engine and copy-out) each return their own cumulative
    long integration."""
    n_ant, n_pol, N, K = 16, 2, 64, 128
    scale = torch.full((N,), 1.0 / 8.0, device=DEV)
    vs = [synth.volt_int8(n_ant, n_pol, N, K, seed=40 + k) for k in range(3)]
    ref = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    want = []
    for v in vs:
        vt = torch.from_numpy(v).to(DEV)
        ref.xengine(ref.fengine(vt, scale))
        want.append(ref.dump().cpu().numpy())
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    vh = [torch.from_numpy(v).pin_memory() for v in vs]
    outs = [torch.zeros((N, c.n_base), dtype=torch.complex128).pin_memory() for _ in vs]
    for k in range(3):
        c.fx_host(vh[k], scale, outs[k])
    torch.cuda.synchronize()
    for k in range(3):
        assert np.array_equal(outs[k].numpy(), want[k]), k
    c.check_status()
    c.close()
    ref.close()


# --------------------------------------------------------------------------- FP16 range: any magnitude
@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("fp16_hilo", 5e-5)])
@pytest.mark.parametrize("mag", [1e-3, 1e3, 1e-6, 1e12])
def test_fp16_paths_hold_their_bound_at_any_magnitude(cuda_ok, prec, tol, mag):
    """The same N(0,1) + sources data scaled by 1e-3, 1e3, 1e-6 and 1e12: without
    range scaling FP16 would round small values into its subnormals (losing the
    hi/lo split's low part) and overflow large ones (above 65504). The per-row
    power-of-two scaling keeps both bounds for any magnitude."""
    n_in, K, n_chan = 200, 264, 2
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=17, src_amp=0.1)
    Xs = (X.astype(np.complex128) * mag).astype(np.complex64)
    c = api.Correlator(n_in, 1, n_chan, K, precision=prec)
    c.xengine(torch.from_numpy(Xs).to(DEV))
    V = c.accum().cpu().numpy().astype(np.complex128)
    c.check_status()
    assert np.all(np.isfinite(V))
    emax, erms = norm_err(V, oracle.cmac(Xs), n_in)
    assert emax <= tol, (prec, mag, emax, erms)
    c.close()


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("fp16_hilo", 5e-5)])
def test_fp16_paths_inputs_of_very_different_magnitudes(cuda_ok, prec, tol):
    """Inputs spanning twelve decades within one channel (input i scaled by
    10^((i mod 13) - 6)), with gains, K not a multiple of 8, and the cross-only
    rectangle: each row gets its own power of two, so every normalised error
    e_ij = |dV_ij| / sqrt(|V_ii| |V_jj|) stays within the bound."""
    n_in, K, n_chan = 150, 93, 2
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=23, src_amp=0.1).astype(np.complex128)
    X *= (10.0 ** ((np.arange(n_in) % 13) - 6))[None, :, None]
    X = X.astype(np.complex64)
    g = synth.gains(n_in, seed=23)
    ref = oracle.apply_gains(oracle.cmac(X), g, n_in)
    c = api.Correlator(n_in, 1, n_chan, K, precision=prec)
    Xt, gt = torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV)
    c.xengine(Xt, gt)
    V = c.accum().cpu().numpy().astype(np.complex128)
    c.check_status()
    emax, erms = norm_err(V, ref, n_in)
    assert emax <= tol, (prec, emax, erms)
    p0, n_p, q0, n_q = 20, 70, 90, 60
    out = c.xengine_cross(Xt, p0, n_p, q0, n_q, gains=gt).cpu().numpy().astype(np.complex128)
    full = oracle.unpack_full(ref, n_in)
    d = np.abs(np.diagonal(full, axis1=1, axis2=2))
    norm = np.sqrt(d[:, p0:p0 + n_p, None] * d[:, None, q0:q0 + n_q])
    assert np.max(np.abs(out - full[:, p0:p0 + n_p, q0:q0 + n_q]) / norm) <= tol
    c.close()


def test_int8_layout_cross_only(cuda_ok):
    """The cross-only rectangle also takes complex int8 channelised data (converted
    to planar codes by the library), bit-exact."""
    n_in, K, n_chan = 140, 72, 2
    X = synth.chan_int8(n_chan, n_in, K, seed=31)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8")
    out = c.xengine_cross(torch.from_numpy(X).to(DEV), 10, 120, 0, 140).cpu().numpy().astype(np.int64)
    Vp = oracle.cmac(X)
    full = oracle.unpack_full(Vp[..., 0] + 1j * Vp[..., 1], n_in)[:, 10:130, 0:140]
    assert np.array_equal(out[..., 0], full.real.astype(np.int64))
    assert np.array_equal(out[..., 1], full.imag.astype(np.int64))
    c.close()
