"""ctypes loader for libcorr.so (the C ABI declared in include/corr.h).

The library is built in-tree by ``paper_1305_5639_gb300.build``. There is no CPU
fallback: if the shared library is missing or cannot be loaded, every entry point
raises."""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcorr.so")

CORR_OK = 0
CORR_EINVAL = 1
CORR_ENOMEM = 2
CORR_ECUDA = 3
CORR_EOVERFLOW = 4
CORR_ESTATE = 5
CORR_ETIMEOUT = 6
CORR_EUNSUPPORTED = 7

PREC = {"fp32": 0, "int8": 1, "fp16": 2, "fp16_hilo": 3}
CORR_FLAG_PLANAR = 1
CORR_FLAG_FUSED_DUMP = 2
CORR_FLAG_FENGINE_CUDACORE = 4
XENG = {"auto": 0, "cudacore": 1, "tcgen05": 2}
STAGES = ("fengine", "pfb", "power", "prep", "xengine", "dump", "adj_prep", "adj_gemm", "adj_reduce")


class corr_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("xengine", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("device", ctypes.c_int32)]


class corr_sub_desc(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_chan", ctypes.c_int32), ("n_spectra", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("planes", ctypes.c_void_p), ("vis", ctypes.c_void_p)]


# (name, restype, argtypes) for every symbol of include/corr.h
_P = ctypes.c_void_p
_S = ctypes.c_int32
SIGNATURES = [
    ("corr_create", _S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                         ctypes.POINTER(corr_opts), ctypes.POINTER(ctypes.c_void_p)]),
    ("corr_destroy", _S, [_P]),
    ("corr_status_str", ctypes.c_char_p, [_S]),
    ("corr_last_error", ctypes.c_char_p, []),
    ("corr_n_baselines", ctypes.c_int64, [_P]),
    ("corr_fengine", _S, [_P, _P, _P, _P, _P]),
    ("corr_fengine_power", _S, [_P, _P, _P, _P]),
    ("corr_set_delays", _S, [_P, _P]),
    ("corr_set_pfb", _S, [_P, ctypes.c_int32, _P]),
    ("corr_xengine", _S, [_P, _P, _P, _P]),
    ("corr_set_short_time", _S, [_P, ctypes.c_int32, _P]),
    ("corr_xengine_cross", _S, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    ("corr_get_accum", _S, [_P, _P, _P]),
    ("corr_dump", _S, [_P, _P, _P]),
    ("corr_flush", _S, [_P, _P]),
    ("corr_restore_vis", _S, [_P, _P, _P]),
    ("corr_selftest_bounded_wait", _S, [ctypes.c_int32, ctypes.c_int64]),
    ("corr_check_status", _S, [_P, _P]),
    ("corr_reset", _S, [_P, _P]),
    ("corr_backward", _S, [_P, _P, _P, _P, _P, _P, _P]),
    ("corr_fengine_power_noalloc", _S, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        _P, _P]),
    ("corr_fx_host", _S, [_P, _P, _P, _P, _P]),
    ("corr_fx_host_accum", _S, [_P, _P, _P, _P, _P]),
    ("corr_set_stage_timing", _S, [_P, ctypes.c_int32]),
    ("corr_stage_times", _S, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    ("corr_batch_create", _S, [ctypes.c_int32, ctypes.POINTER(corr_sub_desc), ctypes.POINTER(corr_opts),
                               ctypes.POINTER(ctypes.c_void_p)]),
    ("corr_batch_tune", _S, [_P, ctypes.c_char_p, _P]),
    ("corr_batch_run", _S, [_P, _P]),
    ("corr_batch_check_status", _S, [_P, _P]),
    ("corr_batch_channels_per_tile", ctypes.c_int32, [_P, ctypes.c_int32]),
    ("corr_batch_destroy", _S, [_P]),
]

_lib = None


class CorrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {status_str(status)}"
        if status == CORR_ECUDA:
            msg += f" [{last_error()}]"
        super().__init__(msg)


def load():
    """Load libcorr.so (raises if it is absent: build it with
    ``python -c 'import __graft_entry__ as g; g.build()'``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcorr.so not built at {LIB_PATH}; run the package build first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_str(s: int) -> str:
    return load().corr_status_str(s).decode()


def last_error() -> str:
    return load().corr_last_error().decode()


def check(status: int, where: str):
    if status != CORR_OK:
        raise CorrError(status, where)
