"""GB300-native FX correlator hot path (Wang & Harris 2013, Section 2).

The compute runs in libcorr.so (hand-written sm_103a CUDA behind the C ABI of
include/corr.h). This package is its thin Python binding (``api``), an
autograd wrapper (``autograd.CorrFn``) and the in-tree build (``build``)."""
from . import _lib  # noqa: F401

__all__ = ["api", "autograd", "build"]


def __getattr__(name):
    if name in ("api", "autograd", "build"):
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
