"""Auxiliary subsystems: checkpoint / resume of the FP64 long integration, and the
device-side bounded-wait self-test (failure detection without a GPU fault)."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api
from paper_1305_5639_gb300._lib import CorrError, CORR_EINVAL

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _planar(X):
    return np.ascontiguousarray(np.transpose(X, (0, 3, 1, 2)).astype(np.float16))


def test_restore_vis_resumes_long_integration(cuda_ok):
    """Two integrations in one handle equal the first dumped, restored into a fresh
    handle, and the second integrated there (exact: integers in FP64)."""
    n_in, K, n_chan = 130, 256, 3
    X1 = synth.chan_int8(n_chan, n_in, K, seed=1)
    X2 = synth.chan_int8(n_chan, n_in, K, seed=2)
    a = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    for X in (X1, X2):
        a.xengine(torch.from_numpy(_planar(X)).to(DEV))
        ref = a.dump()
    b = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    b.xengine(torch.from_numpy(_planar(X1)).to(DEV))
    ckpt = b.dump().clone()
    b.close()
    c = api.Correlator(n_in, 1, n_chan, K, precision="int8", planar=True)
    c.xengine(torch.from_numpy(_planar(X2)).to(DEV))  # an integration in progress is dropped
    c.restore_vis(ckpt)
    c.xengine(torch.from_numpy(_planar(X2)).to(DEV))
    got = c.dump()
    assert torch.equal(got, ref)
    V = oracle.cmac(X1) + oracle.cmac(X2)
    assert np.array_equal(got.cpu().numpy(), V[..., 0] + 1j * V[..., 1])
    c.restore_vis(None)  # zeros
    assert int(c.dump().abs().max().item()) == 0
    with pytest.raises(ValueError):
        c.restore_vis(ckpt[:, 1:])
    a.close()
    c.close()


def test_bounded_wait_selftest_times_out_and_context_survives(cuda_ok):
    limit = 20_000_000  # 20 ms
    t0 = time.perf_counter()
    api.corr_selftest_bounded_wait(0, limit)  # raises unless the wait gave up as designed
    assert time.perf_counter() - t0 >= limit * 1e-9
    for bad in (10, 5_000_000_000):
        with pytest.raises(CorrError) as e:
            api.corr_selftest_bounded_wait(0, bad)
        assert e.value.status == CORR_EINVAL
    # the context is still usable: an exact correlation right after
    X = synth.chan_int8(2, 40, 64, seed=5)
    c = api.Correlator(40, 1, 2, 64, precision="int8", planar=True)
    c.xengine(torch.from_numpy(_planar(X)).to(DEV))
    c.check_status()
    assert np.array_equal(c.accum().cpu().numpy().astype(np.int64), oracle.cmac(X))
    c.close()


def test_stage_timing_counts_and_times_each_stage(cuda_ok):
    """Per-stage event timing (tracing): an FP16 step records the operand conversion,
    the X-engine and the dump separately, one launch each, with positive times;
    reading clears; switched off, launches are still counted but not timed. (Plain
    FP16 dumps at once; the INT8 and hi/lo dumps defer into the next X-engine launch
    and count no dump launch of their own.)"""
    n_in, K, n_chan = 130, 96, 3
    X = torch.from_numpy(synth.chan_sources(n_chan, n_in, K, n_src=2, seed=4, src_amp=0.1)).to(DEV)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16")
    c.set_stage_timing(True)
    for _ in range(2):
        c.xengine(X)
        c.dump(copy=False)
    t = c.stage_times()
    for st in ("prep", "xengine", "dump"):
        assert t[st][1] == 2 and t[st][0] > 0.0, (st, t[st])
    assert t["fengine"] == (0.0, 0)
    assert all(v == (0.0, 0) for v in c.stage_times().values())  # cleared by the read
    c.set_stage_timing(False)
    c.xengine(X)
    t = c.stage_times()
    assert t["xengine"] == (0.0, 1) and t["prep"] == (0.0, 1)
    c.check_status()
    c.close()
    h = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    h.set_stage_timing(True)
    for _ in range(2):
        h.xengine(X)
        h.dump(copy=False)
    t = h.stage_times()
    assert t["xengine"][1] == 2 and t["dump"][1] == 0  # the first dump rode in the second launch
    h.flush()
    assert h.stage_times()["dump"][1] == 1  # the last one, settled by the flush
    h.check_status()
    h.close()
