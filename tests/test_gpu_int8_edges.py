"""The int8 code -128 through every F-engine mode and every INT8 X-engine path.

The paper's streams are 8-bit integers (Section 5), so -128 is a legal sample,
and a legal channelised code for callers who fill the X-engine's input
themselves. It is the one code whose negation is not an int8, and the one that
puts a 512-spectrum FP32 partial (narrow form) or a 1024-spectrum one (wide
form) exactly at 2^24. The workload generators clip at -127; these tests draw
wider noise clipped at -128 (synth's ``lo`` option) and compare bit for bit with
the oracle (Eq. 2 in int64), plus closed forms for constant inputs at the INT32
guard's edge."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"
SIG = 48.0  # about half a percent of the samples land on -128


def _planar(X):
    return np.ascontiguousarray(np.transpose(X, (0, 3, 1, 2)).astype(np.float16))


def _requant_check(out, S, scale, N, taps=1):
    """Codes away from a rounding boundary (beyond the FP32 FFT error) are unique;
    the rest differ by at most one."""
    q, margin = oracle.requant(S, scale)
    eps = 8 * np.log2(N) * max(taps, 1) * 2.0 ** -24 * np.sqrt(np.mean(np.abs(S) ** 2)) * scale.max() * 8
    sure = margin > eps
    assert sure.mean() > 0.9
    assert np.array_equal(out[sure], q[sure])
    assert np.all(np.abs(out.astype(np.int32) - q.astype(np.int32)) <= 1)
    assert out.min() >= -127  # the re-packing clips symmetrically


# --------------------------------------------------------------------------- F-engine
@pytest.mark.parametrize("planar", [False, True])
@pytest.mark.parametrize("N,n_ant,n_pol,K", [(64, 3, 2, 24), (256, 2, 1, 40), (1024, 1, 2, 40)])
def test_fengine_minus128_plain(cuda_ok, planar, N, n_ant, n_pol, K):
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=N + K, sigma=SIG, lo=-128)
    assert (v == -128).any()
    v[0, :N, 0] = -128  # one whole frame's real parts at -128 (all-sums path of the FFT)
    rng = np.random.default_rng(N)
    scale = (rng.uniform(0.8, 1.25, N) * 16.0 / (SIG * np.sqrt(N))).astype(np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=planar)
    out = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    if planar:
        out = np.transpose(out, (0, 2, 3, 1)).astype(np.int8)
    _requant_check(out, oracle.channelise(v, N), scale, N)
    p = c.fengine_power(torch.from_numpy(v).to(DEV)).cpu().numpy()
    assert np.allclose(p, oracle.channel_power(oracle.channelise(v, N)), rtol=1e-4)
    c.close()


@pytest.mark.parametrize("planar", [False, True])
def test_fengine_minus128_delays(cuda_ok, planar):
    N, n_ant, n_pol, K = 256, 2, 2, 24
    n_in = n_ant * n_pol
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=5, sigma=SIG, lo=-128)
    assert (v == -128).any()
    d = np.random.default_rng(3).uniform(-1.5 * N, 1.5 * N, n_in).astype(np.float32)
    d[0] = 0.0
    scale = np.full(N, 16.0 / (SIG * np.sqrt(N)), np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=planar)
    c.set_delays(d)
    out = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    if planar:
        out = np.transpose(out, (0, 2, 3, 1)).astype(np.int8)
    _requant_check(out, oracle.channelise_delayed(v, N, d), scale, N)
    c.close()


def test_fengine_minus128_pfb(cuda_ok):
    N, n_ant, n_pol, K, P = 256, 2, 2, 16, 4
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=8, sigma=SIG, lo=-128)
    assert (v == -128).any()
    x = (np.arange(P * N) - P * N / 2 + 0.5) / N
    h = (np.sinc(x) * np.hanning(P * N)).reshape(P, N).astype(np.float32)
    c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
    c.set_pfb(h)
    S = oracle.channelise_pfb(v, N, h)
    scale = (16.0 / np.sqrt(np.mean(np.abs(S) ** 2, axis=(1, 2)) / 2)).astype(np.float32)
    out = c.fengine(torch.from_numpy(v).to(DEV), torch.from_numpy(scale).to(DEV)).cpu().numpy()
    out = np.transpose(out, (0, 2, 3, 1)).astype(np.int8)
    _requant_check(out, S, scale, N, taps=P)
    c.close()


# --------------------------------------------------------------------------- X-engines, random data with -128
@pytest.mark.parametrize("engine", ["tcgen05", "cudacore"])
@pytest.mark.parametrize("n_in,K,n_chan", [(200, 1032, 2), (70, 37, 3)])
def test_xengine_minus128_int8_layout(cuda_ok, engine, n_in, K, n_chan):
    X = synth.chan_int8(n_chan, n_in, K, seed=n_in + K, sigma=SIG, lo=-128)
    assert (X == -128).any()
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", xengine=engine)
    c.xengine(torch.from_numpy(X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    assert np.array_equal(V, oracle.cmac(X))
    c.close()


@pytest.mark.parametrize("n_in,K,n_chan", [(300, 2048, 2), (130, 1032, 1), (8, 64, 3)])
def test_xengine_minus128_planar_wide(cuda_ok, n_in, K, n_chan):
    X = synth.chan_int8(n_chan, n_in, K, seed=3 * n_in + K, sigma=SIG, lo=-128)
    assert (X == -128).any()
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    c.xengine(torch.from_numpy(_planar(X)).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    assert np.array_equal(V, oracle.cmac(X))
    c.close()


def test_short_time_minus128(cuda_ok):
    n_in, K, n_chan, blk = 140, 1024, 2, 256
    X = synth.chan_int8(n_chan, n_in, K, seed=77, sigma=SIG, lo=-128)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    st = c.set_short_time(blk)
    c.xengine(torch.from_numpy(_planar(X)).to(DEV))
    acc = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    got = st.cpu().numpy().astype(np.int64)
    for b in range(K // blk):
        ref = oracle.cmac(np.ascontiguousarray(X[:, :, b * blk:(b + 1) * blk]))
        assert np.array_equal(got[b], np.transpose(ref, (0, 2, 1))), b
    assert np.array_equal(acc, oracle.cmac(X))
    c.close()


def test_cross_minus128(cuda_ok):
    n_in, K, n_chan = 260, 512, 2
    p0, n_p, q0, n_q = 130, 130, 0, 130
    X = synth.chan_int8(n_chan, n_in, K, seed=91, sigma=SIG, lo=-128)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    out = c.xengine_cross(torch.from_numpy(_planar(X)).to(DEV), p0, n_p, q0, n_q).cpu().numpy().astype(np.int64)
    c.check_status()
    Vp = oracle.cmac(X)
    full = oracle.unpack_full(Vp[..., 0] + 1j * Vp[..., 1], n_in)[:, p0:p0 + n_p, q0:q0 + n_q]
    assert np.array_equal(out[..., 0], full.real.astype(np.int64))
    assert np.array_equal(out[..., 1], full.imag.astype(np.int64))
    c.close()


def test_batch_minus128(cuda_ok):
    shapes = [(40, 3, 512), (130, 2, 1024), (16, 5, 64)]
    Xs = [synth.chan_int8(nc, ni, K, seed=ni + K, sigma=SIG, lo=-128) for ni, nc, K in shapes]
    planes = [torch.from_numpy(_planar(X)).to(DEV) for X in Xs]
    b = api.Batch(planes)
    b.run()
    b.check_status()
    for X, v in zip(Xs, b.vis):
        assert np.array_equal(v.cpu().numpy().astype(np.int64), oracle.cmac(X))
    b.close()


# --------------------------------------------------------------------------- constant -128: FP32 partials at 2^24
@pytest.mark.parametrize("path", ["planar", "tcgen05", "cudacore", "short_time"])
def test_all_minus128_partials_reach_2_24(cuda_ok, path):
    """Every sample -128 - 128j: each product of the wide form's D1, D2 halves is
    +-2^14, so a 1024-spectrum chunk sums to exactly +-2^24 (and a 512-spectrum
    narrow chunk of re re + im im too). Closed form: V_ij = 2^15 K, Im V_ij = 0."""
    n_in, K, n_chan = 136, 2048, 1
    X = np.full((n_chan, n_in, K, 2), -128, np.int8)
    planar = path in ("planar", "short_time")
    eng = "cudacore" if path == "cudacore" else ("auto" if planar else "tcgen05")
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", xengine=eng, planar=planar)
    st = c.set_short_time(512) if path == "short_time" else None
    c.xengine(torch.from_numpy(_planar(X) if planar else X).to(DEV))
    V = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    assert np.all(V[..., 0] == 2 ** 15 * K) and np.all(V[..., 1] == 0)
    if st is not None:
        s = st.cpu().numpy().astype(np.int64)
        assert np.all(s[:, :, 0] == 2 ** 15 * 512) and np.all(s[:, :, 1] == 0)
    c.close()


def test_int32_guard_edge_all_minus128(cuda_ok):
    """The largest integration the INT32 guard admits, n_spectra = 65535 (65528 for
    the planar layout, a multiple of 8), with every sample -128 - 128j: the autos
    reach 2^15 * 65535 = 2^31 - 2^15, still an INT32; one more spectrum is refused."""
    from paper_1305_5639_gb300._lib import CorrError, CORR_EOVERFLOW

    n_in = 8
    for planar, K in ((False, 65535), (True, 65528)):
        X = np.full((1, n_in, K, 2), -128, np.int8)
        c = api.Correlator(n_in, 1, 1, K, precision="int8", planar=planar)
        c.xengine(torch.from_numpy(_planar(X) if planar else X).to(DEV))
        V = c.accum().cpu().numpy().astype(np.int64)
        c.check_status()
        assert np.all(V[..., 0] == 2 ** 15 * K) and np.all(V[..., 1] == 0)
        with pytest.raises(CorrError) as e:  # a second integration would pass 2^31
            c.xengine(torch.from_numpy(_planar(X) if planar else X).to(DEV))
        assert e.value.status == CORR_EOVERFLOW
        c.close()
    with pytest.raises(CorrError) as e:
        api.Correlator(n_in, 1, 1, 65536, precision="int8")
    assert e.value.status == CORR_EOVERFLOW
