"""Cross-only rectangle X-engine (corr_xengine_cross) against the oracle: the
rectangle equals the corresponding block of the full Hermitian matrix built from
the oracle's lower triangle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _planar(X):
    return np.ascontiguousarray(np.transpose(X, (0, 3, 1, 2)).astype(np.float16))


def _full_int(Vp, n_in):
    """[n_chan, B, 2] int64 -> full [n_chan, n_in, n_in] complex (exact integers)."""
    return oracle.unpack_full(Vp[..., 0] + 1j * Vp[..., 1], n_in)


@pytest.mark.parametrize("n_in,K,n_chan,p0,n_p,q0,n_q", [
    (300, 256, 2, 0, 130, 130, 170),     # two disjoint groups, ragged tiles both ways
    (300, 136, 1, 10, 140, 0, 300),      # overlapping ranges: any block of the full matrix
    (64, 64, 3, 40, 24, 0, 40),          # small groups, several channels
    (260, 512, 1, 131, 129, 3, 128),
])
def test_cross_int8_bit_exact(cuda_ok, n_in, K, n_chan, p0, n_p, q0, n_q):
    X = synth.chan_int8(n_chan, n_in, K, seed=p0 + n_q)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    out = c.xengine_cross(torch.from_numpy(_planar(X)).to(DEV), p0, n_p, q0, n_q)
    c.check_status()
    got = out.cpu().numpy().astype(np.int64)
    full = _full_int(oracle.cmac(X), n_in)[:, p0:p0 + n_p, q0:q0 + n_q]
    assert np.array_equal(got[..., 0], full.real.astype(np.int64))
    assert np.array_equal(got[..., 1], full.imag.astype(np.int64))
    # the handle's accumulator is untouched
    assert int(c.accum().abs().max()) == 0
    c.close()


@pytest.mark.parametrize("prec,tol", [("fp16", 2e-3), ("fp16_hilo", 5e-5)])
def test_cross_fp16_with_gains(cuda_ok, prec, tol):
    n_in, K, n_chan = 200, 136, 2
    p0, n_p, q0, n_q = 150, 50, 0, 150
    X = synth.chan_sources(n_chan, n_in, K, n_src=3, seed=12, src_amp=0.1)
    g = synth.gains(n_in, seed=12)
    c = api.Correlator(n_in, 1, n_chan, K, precision=prec)
    out = c.xengine_cross(torch.from_numpy(X).to(DEV), p0, n_p, q0, n_q, gains=torch.from_numpy(g).to(DEV))
    c.check_status()
    got = out.cpu().numpy().astype(np.complex128)
    full = oracle.unpack_full(oracle.apply_gains(oracle.cmac(X), g, n_in), n_in)
    ref = full[:, p0:p0 + n_p, q0:q0 + n_q]
    d = np.abs(np.diagonal(full, axis1=1, axis2=2))  # |V_ii|
    norm = np.sqrt(d[:, p0:p0 + n_p, None] * d[:, None, q0:q0 + n_q])
    assert np.max(np.abs(got - ref) / norm) <= tol
    c.close()


def test_cross_validation(cuda_ok):
    from paper_1305_5639_gb300._lib import CorrError, CORR_EINVAL, CORR_EUNSUPPORTED

    n_in, K = 40, 64
    X = torch.zeros((1, 2, n_in, K), dtype=torch.float16, device=DEV)
    c = api.Correlator(n_in, 1, 1, K, precision="int8", planar=True)
    for args in ((0, 41, 0, 1), (-1, 2, 0, 1), (0, 1, 39, 2), (0, 0, 0, 1)):
        with pytest.raises(CorrError) as e:
            c.xengine_cross(X, *args)
        assert e.value.status == CORR_EINVAL, args
    c.close()
    # the rectangle runs on the tensor-core X-engine only
    for kw in (dict(precision="int8", xengine="cudacore"), dict(precision="fp32")):
        c = api.Correlator(n_in, 1, 1, K, **kw)
        with pytest.raises(CorrError) as e:
            c.xengine_cross(torch.zeros((1, n_in, K, 2), dtype=torch.int8, device=DEV), 0, 8, 8, 8)
        assert e.value.status == CORR_EUNSUPPORTED, kw
        c.close()
