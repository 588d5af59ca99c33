"""Deferred integration dumps on the tensor-core X-engine (INT8 and FP16 hi/lo).

corr_dump without an output copy keeps the finished accumulator aside and the
next X-engine launch adds it into the FP64 long integration from otherwise idle
warps; corr_flush, corr_dump with an output, corr_fx_host, corr_restore_vis and
corr_reset settle or drop it. Every observable result must equal the immediate
dump's, bit for bit, and the oracle's sum of integrations."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"
SIG8 = 48.0  # wide int8 noise, clipped at -128


def _planar(X):
    return np.ascontiguousarray(np.transpose(X, (0, 3, 1, 2)).astype(np.float16))


def _c(V):
    return V[..., 0] + 1j * V[..., 1]


@pytest.mark.parametrize("planar", [True, False])
def test_deferred_dumps_equal_oracle_sum(cuda_ok, planar):
    n_in, K, n_chan = 200, 256, 3
    parts = [synth.chan_int8(n_chan, n_in, K, seed=50 + t) for t in range(4)]
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=planar)
    for t, X in enumerate(parts):
        c.xengine(torch.from_numpy(_planar(X) if planar else X).to(DEV))
        # the accumulator holds this integration alone, whatever is pending
        assert np.array_equal(c.accum().cpu().numpy().astype(np.int64), oracle.cmac(X)), t
        c.dump(copy=False)  # deferred into the next X-engine launch
        assert int(c.accum().abs().max()) == 0  # logically clear after the dump
    vis = c.dump().cpu().numpy()  # settles the last deferred dump, then copies
    c.check_status()
    want = oracle.dump([oracle.cmac(X) for X in parts])
    assert np.array_equal(vis, _c(want))
    c.close()


def test_flush_and_repeated_dump_calls(cuda_ok):
    n_in, K, n_chan = 130, 128, 2
    parts = [synth.chan_int8(n_chan, n_in, K, seed=60 + t) for t in range(3)]
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    out = torch.empty((n_chan, n_in * (n_in + 1) // 2), dtype=torch.complex128, device=DEV)
    c.xengine(torch.from_numpy(_planar(parts[0])).to(DEV))
    c.dump(copy=False)
    c.dump(copy=False)  # nothing accumulated since: no second dump
    c.flush()
    c.flush()  # nothing pending: no-op
    api.corr_dump(c.h, out)
    assert np.array_equal(out.cpu().numpy(), _c(oracle.cmac(parts[0])))
    # two X-engine calls in one integration, then a deferred dump and a flush
    c.xengine(torch.from_numpy(_planar(parts[1])).to(DEV))
    c.xengine(torch.from_numpy(_planar(parts[2])).to(DEV))
    c.dump(copy=False)
    c.flush()
    api.corr_dump(c.h, out)
    c.check_status()
    want = oracle.dump([oracle.cmac(X) for X in parts])
    assert np.array_equal(out.cpu().numpy(), _c(want))
    c.close()


def test_restore_and_reset_drop_a_pending_dump(cuda_ok):
    n_in, K, n_chan = 64, 64, 2
    X1 = synth.chan_int8(n_chan, n_in, K, seed=71)
    X2 = synth.chan_int8(n_chan, n_in, K, seed=72)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    c.xengine(torch.from_numpy(_planar(X1)).to(DEV))
    saved = c.dump()  # checkpoint: integration 1
    c.xengine(torch.from_numpy(_planar(X2)).to(DEV))
    c.dump(copy=False)  # integration 2 pending
    c.restore_vis(saved)  # resume from the checkpoint: integration 2's dump is dropped
    c.xengine(torch.from_numpy(_planar(X2)).to(DEV))  # no pending dump rides along
    vis = c.dump().cpu().numpy()
    assert np.array_equal(vis, _c(oracle.dump([oracle.cmac(X1), oracle.cmac(X2)])))
    c.xengine(torch.from_numpy(_planar(X1)).to(DEV))
    c.dump(copy=False)
    c.reset()  # everything zero, the pending dump dropped
    c.xengine(torch.from_numpy(_planar(X2)).to(DEV))
    vis = c.dump().cpu().numpy()
    c.check_status()
    assert np.array_equal(vis, _c(oracle.cmac(X2)))
    c.close()


def test_deferred_dump_with_short_time_output_and_fx_host(cuda_ok):
    """The deferred dump also rides in the short-time X-engine launch, and the host
    pipeline settles a pending dump before its own: the long integration equals that
    of a handle making the same calls with immediate dumps, bit for bit, and its
    X-engine part the oracle's."""
    n_ant, n_pol, N, K = 8, 2, 64, 128
    n_in = n_ant * n_pol
    X = synth.chan_int8(N, n_in, K, seed=81)
    v = synth.volt_int8(n_ant, n_pol, N, K, seed=82)
    scale = torch.full((N,), 1.0 / 8.0, device=DEV)
    res = []
    for deferred in (True, False):
        c = api.Correlator(n_ant, n_pol, N, K, precision="int8", planar=True)
        settle = (lambda: c.dump(copy=False)) if deferred else (lambda: c.dump())
        st = c.set_short_time(64)
        c.xengine(torch.from_numpy(_planar(X)).to(DEV))
        settle()
        c.xengine(torch.from_numpy(_planar(X)).to(DEV))  # short-time launch carries the dump
        c.set_short_time(out=False)
        del st
        settle()  # pending again (deferred)
        two = c.dump().cpu().numpy()  # settles: the two X-engine integrations
        assert np.array_equal(two, _c(oracle.dump([oracle.cmac(X), oracle.cmac(X)])))
        c.xengine(torch.from_numpy(_planar(X)).to(DEV))
        settle()  # a third, pending when the host pipeline starts (deferred)
        vis_h = torch.empty((N, n_in * (n_in + 1) // 2), dtype=torch.complex128).pin_memory()
        c.fx_host(torch.from_numpy(v).pin_memory(), scale, vis_h)
        torch.cuda.synchronize()
        c.check_status()
        res.append(vis_h.numpy().copy())
        c.close()
    assert np.array_equal(res[0], res[1])


def test_deferred_hilo_dumps_equal_immediate_ones(cuda_ok):
    """FP16 hi/lo also defers: the FP64 sums equal those of a handle that dumps at
    once (each dump with an output copy) bit for bit, and the oracle's within 5e-5."""
    n_in, K, n_chan = 150, 136, 2
    parts = [synth.chan_sources(n_chan, n_in, K, n_src=3, seed=90 + t, src_amp=0.1) for t in range(3)]
    a = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    b = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    out = torch.empty((n_chan, n_in * (n_in + 1) // 2), dtype=torch.complex128, device=DEV)
    for X in parts:
        Xt = torch.from_numpy(X).to(DEV)
        a.xengine(Xt)
        a.dump(copy=False)  # deferred
        b.xengine(Xt)
        api.corr_dump(b.h, out)  # immediate (an output copy settles it at once)
    va, vb = a.dump().cpu().numpy(), b.dump().cpu().numpy()
    a.check_status()
    b.check_status()
    assert np.array_equal(va, vb)
    ref = oracle.dump([oracle.cmac(X) for X in parts])
    i, j = oracle.tri_pairs(n_in)
    aut = np.abs(ref[..., oracle.packed_index(np.arange(n_in), np.arange(n_in))])
    e = np.abs(va - ref) / np.sqrt(aut[..., i] * aut[..., j])
    assert e.max() <= 5e-5
    a.close()
    b.close()


def _vis0(rng, n_chan, B, integer):
    """A starting long integration: integer-valued doubles up to 2^40 (INT8 sums add in
    integers), with some non-integers, some beyond 2^52 (both take the FP64 add), and
    zeros; or, for FP32 sums, doubles of mixed magnitude."""
    if integer:
        re = rng.integers(-2 ** 40, 2 ** 40, (n_chan, B)).astype(np.float64)
        im = rng.integers(-2 ** 40, 2 ** 40, (n_chan, B)).astype(np.float64)
        m = rng.random((n_chan, B))
        re[m < 0.05] += 0.5
        im[(m > 0.05) & (m < 0.1)] = 2.0 ** 53 + 2.0 * rng.integers(0, 1000, ((m > 0.05) & (m < 0.1)).sum())
        re[m > 0.95] = 0.0
        im[m > 0.97] = -0.0
    else:
        re = rng.standard_normal((n_chan, B)) * 10.0 ** rng.integers(-6, 9, (n_chan, B))
        im = rng.standard_normal((n_chan, B)) * 10.0 ** rng.integers(-6, 9, (n_chan, B))
        re[rng.random((n_chan, B)) < 0.03] = 0.0
    return re + 1j * im


@pytest.mark.parametrize("precision", ["int8", "fp16", "fp16_hilo"])
@pytest.mark.parametrize("mode", ["immediate", "deferred"])
def test_dump_add_is_the_fp64_add(cuda_ok, precision, mode):
    """Property of the dump, whatever form it takes: the long integration becomes
    vis0 + acc, each part one IEEE FP64 addition of the accumulator's value (for INT8
    the oracle's exact sums; for FP32 sums the accumulator read back) to the starting
    value, bit for bit (the integer forms of the conversion and of the INT8 add must
    agree with it everywhere, including zeros, non-integers and values beyond 2^52)."""
    n_in, K, n_chan = 136, 136, 2
    B = n_in * (n_in + 1) // 2
    rng = np.random.default_rng(7)
    if precision == "int8":
        X = synth.chan_int8(n_chan, n_in, K, seed=5, sigma=SIG8, lo=-128)
        Xt = torch.from_numpy(_planar(X)).to(DEV)
        c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    else:
        X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=5, src_amp=0.1)
        Xt = torch.from_numpy(X).to(DEV)
        c = api.Correlator(n_in, 1, n_chan, K, precision=precision)
    vis0 = _vis0(rng, n_chan, B, precision == "int8")
    c.restore_vis(torch.from_numpy(vis0).to(DEV))
    c.xengine(Xt)
    if precision == "int8":
        acc = oracle.cmac(X).astype(np.float64)
    else:
        a = c.accum().cpu().numpy()  # complex64: the FP32 sums
        acc = np.stack([a.real, a.imag], axis=-1).astype(np.float64)  # widened exactly
    if mode == "deferred":
        c.dump(copy=False)
        c.xengine(Xt)  # carries the deferred add (INT8 and hi/lo; plain FP16 may not defer)
        vis = c.dump().cpu().numpy()
        want_re = (vis0.real + acc[..., 0]) + acc[..., 0]
        want_im = (vis0.imag + acc[..., 1]) + acc[..., 1]
    else:
        vis = c.dump().cpu().numpy()
        want_re, want_im = vis0.real + acc[..., 0], vis0.imag + acc[..., 1]
    c.check_status()
    assert np.array_equal(vis.real.view(np.int64), want_re.view(np.int64))
    assert np.array_equal(vis.imag.view(np.int64), want_im.view(np.int64))
    c.close()


@pytest.mark.parametrize("precision", ["int8", "fp16", "fp16_hilo"])
def test_fused_dump_add_equals_separate_dump(cuda_ok, precision):
    """The fused form (the X-engine's epilogue adds into the FP64 buffer) gives the same
    bits as the separate dump from the same starting long integration."""
    n_in, K, n_chan = 136, 136, 2
    B = n_in * (n_in + 1) // 2
    vis0 = _vis0(np.random.default_rng(11), n_chan, B, precision == "int8")
    if precision == "int8":
        X = synth.chan_int8(n_chan, n_in, K, seed=6, sigma=SIG8, lo=-128)
        Xt = torch.from_numpy(_planar(X)).to(DEV)
        kw = dict(precision="int8", planar=True)
    else:
        Xt = torch.from_numpy(synth.chan_sources(n_chan, n_in, K, n_src=3, seed=6, src_amp=0.1)).to(DEV)
        kw = dict(precision=precision)
    out = []
    for fused in (False, True):
        c = api.Correlator(n_in, 1, n_chan, K, fused_dump=fused, **kw)
        c.restore_vis(torch.from_numpy(vis0).to(DEV))
        c.xengine(Xt)
        out.append(c.dump().cpu().numpy())
        c.check_status()
        c.close()
    assert np.array_equal(out[0].view(np.int64), out[1].view(np.int64))
