"""The allocation-free power pass (corr_fengine_power_noalloc) against the
handle-based corr_fengine_power, through the C ABI.

The entry point exists for callers that cannot allocate device memory (a host
that owns all device memory up front, or code where an allocation's implicit
synchronisation is not acceptable); its scratch is a static device array shared
by every call, so the test runs it twice in a row on different inputs to show
that each call starts from cleared accumulators. Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth
from paper_1305_5639_gb300._lib import CORR_EINVAL, CORR_OK


def _lib():
    from paper_1305_5639_gb300 import _lib

    return _lib.load()


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    lib = _lib()
    dummy = ctypes.c_void_p(16)
    # 4096 channels would need more than the 1024 FP64 accumulators it holds
    assert lib.corr_fengine_power_noalloc(dummy, 4, 4096, 8, 1, dummy, None) == CORR_EINVAL
    assert b"1024-channel static scratch" in lib.corr_last_error()
    assert lib.corr_fengine_power_noalloc(None, 4, 256, 8, 1, dummy, None) == CORR_EINVAL
    assert b"null" in lib.corr_last_error()
    # more inputs than the F-engine grid holds: a clean argument error, not a launch failure
    assert lib.corr_fengine_power_noalloc(dummy, 65536, 256, 8, 1, dummy, None) == CORR_EINVAL
    assert b"65535" in lib.corr_last_error()
    # precision and alignment rejections carry their own message
    assert lib.corr_fengine_power_noalloc(dummy, 4, 256, 8, 2, dummy, None) == CORR_EINVAL
    assert b"precision" in lib.corr_last_error()
    assert lib.corr_fengine_power_noalloc(ctypes.c_void_p(24), 4, 256, 8, 1, dummy, None) == CORR_EINVAL
    assert b"aligned" in lib.corr_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,N", [("int8", 1024), ("fp32", 256)])
def test_noalloc_power_matches_handle_path_two_calls(cuda_ok, precision, N):
    import torch
    from paper_1305_5639_gb300 import api

    lib = _lib()
    n_ant, n_pol, K = 3, 2, 40
    n_in = n_ant * n_pol
    prec = 1 if precision == "int8" else 0
    c = api.Correlator(n_ant, n_pol, N, K, precision=precision)
    stream = torch.cuda.current_stream()
    for seed in (1, 2):  # two calls in a row share the static scratch
        if precision == "int8":
            v = synth.volt_int8(n_ant, n_pol, N, K, seed=seed)
        else:
            v = synth.volt_fp32(n_in, N, K, seed=seed)
        volt = torch.from_numpy(v).cuda()
        out = torch.full((N,), -1.0, dtype=torch.float32, device="cuda")
        st = lib.corr_fengine_power_noalloc(ctypes.c_void_p(volt.data_ptr()), n_in, N, K, prec,
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == CORR_OK
        ref = c.fengine_power(volt)
        torch.cuda.synchronize()
        assert np.allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-4, atol=0)
    c.close()
