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
    o = corr_opts(0, 0, 4, -1)  # unknown flag bit
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EINVAL
    o = corr_opts(0, 0, 1, -1)  # the planar layout is INT8 only
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    o = corr_opts(1, 0, 1, -1)  # ... and needs n_spectra % 8 == 0
    assert lib.corr_create(4, 1, 16, 12, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    o = corr_opts(1, 0, 2, -1)  # the fused dump needs the planar X-engine
    assert lib.corr_create(4, 1, 16, 16, ctypes.byref(o), ctypes.byref(h)) == CORR_EUNSUPPORTED
    # INT8 guard: n_spectra * 2 * 127^2 must stay below 2^31 (66573 spectra is the first to fail)
    o = corr_opts(1, 0, 0, -1)
    assert lib.corr_create(4, 1, 16, 66573, ctypes.byref(o), ctypes.byref(h)) == CORR_EOVERFLOW
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
    assert lib.corr_n_baselines(None) == -1


def test_int8_guard_boundary_is_exact():
    # largest allowed n_spectra: 2 * 127^2 * n < 2^31
    n = (2**31 - 1) // (2 * 127 * 127)
    assert n == 66572 and 2 * 127 * 127 * n < 2**31 <= 2 * 127 * 127 * (n + 1)
