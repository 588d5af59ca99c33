"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point declared in include/corr.h, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_5639_gb300 import build, _lib

    build.build()
    return _lib.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"CORR_API[^;]*?\b(corr_\w+)\s*\(", txt, flags=re.S))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"corr_create", "corr_fengine", "corr_xengine", "corr_dump", "corr_backward"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_every_symbol(lib):
    from paper_1305_5639_gb300 import _lib, api

    bound = {n for n, _, _ in _lib.SIGNATURES}
    assert _declared() <= bound | {n for n in dir(api) if n.startswith("corr_")}


def test_status_strings(lib):
    from paper_1305_5639_gb300 import _lib

    for code in range(8):
        s = _lib.status_str(code)
        assert s.startswith("CORR_")
    assert _lib.status_str(0) == "CORR_OK"
    assert "unknown" in _lib.status_str(99)


def test_create_rejects_bad_arguments_without_device(lib):
    from paper_1305_5639_gb300._lib import corr_opts, CORR_EINVAL, CORR_EOVERFLOW, CORR_EUNSUPPORTED

    h = ctypes.c_void_p()
    assert lib.corr_create(0, 1, 16, 16, None, ctypes.byref(h)) == CORR_EINVAL
    assert lib.corr_create(4, 1, 16, 0, None, ctypes.byref(h)) == CORR_EINVAL
    assert lib.corr_create(4, 1, 16, 16, None, None) == CORR_EINVAL
    o = corr_opts(9, 0, 0, -1)
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EINVAL
    o = corr_opts(0, 0, 8, -1)  # unknown flag bit
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EINVAL
    o = corr_opts(0, 0, 1, -1)  # the planar layout is INT8 only
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    o = corr_opts(1, 0, 1, -1)  # ... and needs n_spectra % 8 == 0
    assert lib.corr_create(4, 1, 16, 12, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    o = corr_opts(1, 1, 2, -1)  # the fused dump needs the tensor-core X-engine
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    o = corr_opts(0, 2, 0, -1)  # FP32 has no tensor-core X-engine
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    # INT8 guard: n_spectra * 2 * 128^2 must stay below 2^31 (int8 codes include -128;
    # 65536 spectra is the first to fail)
    o = corr_opts(1, 0, 0, -1)
    assert lib.corr_create(4, 1, 16, 65536, ctypes.byref(o), ctypes.byref(h)) == CORR_EOVERFLOW
    # at most 65535 inputs (one F-engine grid row per input)
    assert lib.corr_create(65536, 1, 16, 16, None, ctypes.byref(h)) == CORR_EINVAL
    assert b"65535" in lib.corr_last_error()
    o = corr_opts(2, 1, 0, -1)  # FP16 has no CUDA-core X-engine
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    assert not h.value


def test_null_handle_calls(lib):
    from paper_1305_5639_gb300._lib import CORR_EINVAL, CORR_OK

    assert lib.corr_destroy(None) == CORR_OK
    assert lib.corr_fengine(None, None, None, None, None) == CORR_EINVAL
    assert lib.corr_xengine(None, None, None, None) == CORR_EINVAL
    assert lib.corr_dump(None, None, None) == CORR_EINVAL
    assert lib.corr_backward(None, None, None, None, None, None, None) == CORR_EINVAL
    assert lib.corr_fx_host(None, None, None, None, None) == CORR_EINVAL
    assert lib.corr_fx_host_accum(None, None, None, None, None) == CORR_EINVAL
    assert lib.corr_n_baselines(None) == -1
    assert lib.corr_set_stage_timing(None, 1) == CORR_EINVAL
    assert lib.corr_stage_times(None, None, None) == CORR_EINVAL


def test_int8_guard_boundary_is_exact():
    # largest allowed n_spectra: 2 * 128^2 * n < 2^31 (an autocorrelation of -128 samples)
    n = (2**31 - 1) // (2 * 128 * 128)
    assert n == 65535 and 2 * 128 * 128 * n < 2**31 <= 2 * 128 * 128 * (n + 1)


def test_batch_create_rejects_bad_arguments_without_device(lib):
    from paper_1305_5639_gb300._lib import (corr_opts, corr_sub_desc, CORR_EINVAL, CORR_EOVERFLOW,
                                            CORR_EUNSUPPORTED)

    b = ctypes.c_void_p()
    fake = 1 << 20  # 16-byte aligned stand-in addresses: never dereferenced before the checks fail
    arr = (corr_sub_desc * 1)(corr_sub_desc(64, 4, 64, 0, fake, fake))
    assert lib.corr_batch_create(0, arr, None, ctypes.byref(b)) == CORR_EINVAL
    assert lib.corr_batch_create(1, arr, None, None) == CORR_EINVAL
    o = corr_opts(0, 0, 0, -1)  # FP32 is not batched
    assert lib.corr_batch_create(1, arr, ctypes.byref(o), ctypes.byref(b)) == CORR_EUNSUPPORTED
    o = corr_opts(1, 1, 0, -1)  # nor is the CUDA-core X-engine
    assert lib.corr_batch_create(1, arr, ctypes.byref(o), ctypes.byref(b)) == CORR_EUNSUPPORTED
    bad = (corr_sub_desc * 1)(corr_sub_desc(64, 4, 65536, 0, fake, fake))  # INT32 guard with -128
    assert lib.corr_batch_create(1, bad, None, ctypes.byref(b)) == CORR_EOVERFLOW
    bad = (corr_sub_desc * 1)(corr_sub_desc(64, 4, 60, 0, fake, fake))  # spectra not a multiple of 8
    assert lib.corr_batch_create(1, bad, None, ctypes.byref(b)) == CORR_EUNSUPPORTED
    assert not b.value
