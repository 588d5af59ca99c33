"""Short-time visibilities (transient-detector hook) from the INT8 tensor-core
X-engine: each block of spectra equals the oracle's correlation of that block alone
(bit-exact), and the blocks sum to the integration."""
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


@pytest.mark.parametrize("n_in,K,n_chan,block", [(300, 1024, 2, 512), (130, 384, 3, 64), (64, 512, 1, 128)])
def test_short_time_blocks_bit_exact(cuda_ok, n_in, K, n_chan, block):
    X = synth.chan_int8(n_chan, n_in, K, seed=n_in + block)
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    st = c.set_short_time(block)
    c.xengine(torch.from_numpy(_planar(X)).to(DEV))
    acc = c.accum().cpu().numpy().astype(np.int64)
    c.check_status()
    got = st.cpu().numpy().astype(np.int64)  # [n_blocks, n_chan, 2, B]
    assert got.shape == (K // block, n_chan, 2, n_in * (n_in + 1) // 2)
    for b in range(K // block):
        ref = oracle.cmac(np.ascontiguousarray(X[:, :, b * block:(b + 1) * block]))  # [n_chan, B, 2]
        assert np.array_equal(got[b], np.transpose(ref, (0, 2, 1))), b
    # the integration is the sum of its blocks
    assert np.array_equal(got.sum(axis=0), np.transpose(acc, (0, 2, 1)))
    # switching the output off leaves the buffer alone
    c.set_short_time(out=False)
    before = st.clone()
    c.xengine(torch.from_numpy(_planar(X)).to(DEV))
    torch.cuda.synchronize()
    assert torch.equal(st, before)
    c.close()


def test_short_time_validation(cuda_ok):
    from paper_1305_5639_gb300._lib import CorrError, CORR_EINVAL, CORR_EUNSUPPORTED

    c = api.Correlator(16, 1, 2, 256, precision="int8", planar=True)
    for blk in (32, 96, 1024, 192):  # not a multiple of 64 in [64, 512] dividing 256
        with pytest.raises(CorrError) as e:
            c.set_short_time(blk, out=torch.zeros(1024, dtype=torch.int32, device=DEV))
        assert e.value.status == CORR_EINVAL, blk
    c.close()
    c = api.Correlator(16, 1, 2, 256, precision="int8")  # not planar
    with pytest.raises(CorrError) as e:
        c.set_short_time(64)
    assert e.value.status == CORR_EUNSUPPORTED
    c.close()
