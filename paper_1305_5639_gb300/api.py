"""Thin Python binding of the libcorr C ABI (include/corr.h), same names.

Only argument marshalling happens here: tensors are passed as raw device pointers
and the CUDA stream defaults to torch's current stream. Every step of the
correlator runs in the library's kernels.

Tensor conventions (all on the handle's CUDA device, contiguous):
  complex int8   -> torch.int8 with a trailing dimension of 2 (re, im)
  complex float  -> torch.complex64, or torch.float32 with a trailing 2
  complex double -> torch.complex128, or torch.float64 with a trailing 2
"""
from __future__ import annotations

import ctypes

import numpy as np

import torch

from . import _lib
from ._lib import PREC, XENG, CorrError, check, corr_opts  # noqa: F401


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not t.is_cuda:
        raise ValueError("libcorr takes device tensors")
    if not t.is_contiguous():
        raise ValueError("libcorr takes contiguous tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def corr_create(n_ant: int, n_pol: int, n_chan: int, n_spectra: int, precision="fp32", xengine="auto",
                device: int = -1, flags: int = 0) -> ctypes.c_void_p:
    lib = _lib.load()
    o = corr_opts(PREC[precision] if isinstance(precision, str) else int(precision),
                  XENG[xengine] if isinstance(xengine, str) else int(xengine), int(flags), int(device))
    h = ctypes.c_void_p()
    check(lib.corr_create(n_ant, n_pol, n_chan, n_spectra, ctypes.byref(o), ctypes.byref(h)), "corr_create")
    return h


def corr_destroy(h) -> None:
    check(_lib.load().corr_destroy(h), "corr_destroy")


def corr_n_baselines(h) -> int:
    return int(_lib.load().corr_n_baselines(h))


def corr_fengine(h, volt, chan_scale, chan_out, stream=None) -> None:
    check(_lib.load().corr_fengine(h, _ptr(volt), _ptr(chan_scale), _ptr(chan_out), _stream(stream)),
          "corr_fengine")


def corr_fengine_power(h, volt, power, stream=None) -> None:
    check(_lib.load().corr_fengine_power(h, _ptr(volt), _ptr(power), _stream(stream)), "corr_fengine_power")


def corr_fengine_power_noalloc(volt, n_in: int, n_chan: int, n_spectra: int, precision, power,
                               stream=None) -> None:
    """Per-channel power pass that allocates no device memory (no handle)."""
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    check(_lib.load().corr_fengine_power_noalloc(_ptr(volt), n_in, n_chan, n_spectra, prec, _ptr(power),
                                                 _stream(stream)), "corr_fengine_power_noalloc")


def _hptr(t):
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
        raise ValueError("corr_fx_host takes contiguous host tensors")
    return ctypes.c_void_p(t.data_ptr())


def corr_fx_host(h, volt_host, chan_scale, vis_host, stream=None) -> None:
    check(_lib.load().corr_fx_host(h, _hptr(volt_host), _ptr(chan_scale), _hptr(vis_host), _stream(stream)),
          "corr_fx_host")


def corr_fx_host_accum(h, volt_host, chan_scale, acc_host, stream=None) -> None:
    check(_lib.load().corr_fx_host_accum(h, _hptr(volt_host), _ptr(chan_scale), _hptr(acc_host), _stream(stream)),
          "corr_fx_host_accum")


def corr_xengine(h, chan_in, gains=None, stream=None) -> None:
    check(_lib.load().corr_xengine(h, _ptr(chan_in), _ptr(gains), _stream(stream)), "corr_xengine")


def corr_get_accum(h, out, stream=None) -> None:
    check(_lib.load().corr_get_accum(h, _ptr(out), _stream(stream)), "corr_get_accum")


def corr_dump(h, vis_out=None, stream=None) -> None:
    check(_lib.load().corr_dump(h, _ptr(vis_out), _stream(stream)), "corr_dump")


def corr_flush(h, stream=None) -> None:
    check(_lib.load().corr_flush(h, _stream(stream)), "corr_flush")


def corr_restore_vis(h, vis_in=None, stream=None) -> None:
    check(_lib.load().corr_restore_vis(h, _ptr(vis_in), _stream(stream)), "corr_restore_vis")


def corr_selftest_bounded_wait(device: int = 0, limit_ns: int = 20_000_000) -> None:
    """Run the device-side bounded-wait self-test (raises CorrError if it fails)."""
    check(_lib.load().corr_selftest_bounded_wait(int(device), int(limit_ns)), "corr_selftest_bounded_wait")


def corr_check_status(h, stream=None) -> None:
    check(_lib.load().corr_check_status(h, _stream(stream)), "corr_check_status")


def corr_reset(h, stream=None) -> None:
    check(_lib.load().corr_reset(h, _stream(stream)), "corr_reset")


def corr_backward(h, grad_vis, chan_in, gains=None, grad_chan=None, grad_gains=None, stream=None) -> None:
    check(_lib.load().corr_backward(h, _ptr(grad_vis), _ptr(chan_in), _ptr(gains), _ptr(grad_chan),
                                    _ptr(grad_gains), _stream(stream)), "corr_backward")


class Correlator:
    """Owns one libcorr handle; allocates outputs as torch tensors."""

    def __init__(self, n_ant: int, n_pol: int, n_chan: int, n_spectra: int, precision="fp32", xengine="auto",
                 device=None, planar: bool = False, fused_dump: bool = False, fengine: str = "auto"):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else int(device))
        self.device = dev
        self.n_ant, self.n_pol, self.n_chan, self.n_spectra = n_ant, n_pol, n_chan, n_spectra
        self.n_in = n_ant * n_pol
        self.precision = precision
        self.planar = planar
        with torch.cuda.device(dev):
            if fengine not in ("auto", "cudacore"):
                raise ValueError("fengine must be 'auto' (tensor cores where they apply) or 'cudacore'")
            flags = ((_lib.CORR_FLAG_PLANAR if planar else 0) | (_lib.CORR_FLAG_FUSED_DUMP if fused_dump else 0)
                     | (_lib.CORR_FLAG_FENGINE_CUDACORE if fengine == "cudacore" else 0))
            self.h = corr_create(n_ant, n_pol, n_chan, n_spectra, precision, xengine, dev.index, flags)
        self.n_base = corr_n_baselines(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            corr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers
    def chan_buffer(self):
        if self.planar:
            return torch.empty((self.n_chan, 2, self.n_in, self.n_spectra), dtype=torch.float16, device=self.device)
        if self.precision == "int8":
            return torch.empty((self.n_chan, self.n_in, self.n_spectra, 2), dtype=torch.int8, device=self.device)
        return torch.empty((self.n_chan, self.n_in, self.n_spectra), dtype=torch.complex64, device=self.device)

    def accum_buffer(self):
        if self.precision == "int8":
            return torch.empty((self.n_chan, self.n_base, 2), dtype=torch.int32, device=self.device)
        return torch.empty((self.n_chan, self.n_base), dtype=torch.complex64, device=self.device)

    # -- calls
    def fengine(self, volt, chan_scale=None, out=None, stream=None):
        out = self.chan_buffer() if out is None else out
        corr_fengine(self.h, volt, chan_scale, out, stream)
        return out

    def fengine_power(self, volt, out=None, stream=None):
        out = torch.empty(self.n_chan, dtype=torch.float32, device=self.device) if out is None else out
        corr_fengine_power(self.h, volt, out, stream)
        return out

    def xengine(self, chan_in, gains=None, stream=None):
        corr_xengine(self.h, chan_in, gains, stream)

    def fx_host(self, volt_host, chan_scale, vis_host, stream=None):
        """Whole step from host buffers (pipelined copies); see corr_fx_host."""
        corr_fx_host(self.h, volt_host, chan_scale, vis_host, stream)

    def fx_host_accum(self, volt_host, chan_scale, acc_host, stream=None):
        """Whole step from host buffers, this integration's INT32 visibilities out
        ([n_chan][B][2] int32 host tensor); see corr_fx_host_accum."""
        corr_fx_host_accum(self.h, volt_host, chan_scale, acc_host, stream)

    def set_pfb(self, window=None):
        """Polyphase filter-bank window [n_taps, n_chan] (float) for the F-engine, or
        None to switch the filter bank off."""
        if window is None:
            check(_lib.load().corr_set_pfb(self.h, 0, None), "corr_set_pfb")
            return
        w = np.ascontiguousarray(np.asarray(window, dtype=np.float32))
        if w.ndim != 2 or w.shape[1] != self.n_chan:
            raise ValueError(f"window must be [n_taps, {self.n_chan}]")
        check(_lib.load().corr_set_pfb(self.h, int(w.shape[0]), w.ctypes.data), "corr_set_pfb")

    def set_short_time(self, block_spectra: int = 512, out=None):
        """Short-time visibilities of every block of `block_spectra` spectra, written by
        each X-engine call into `out` ([n_spectra / block, n_chan, 2, B] int32, allocated
        if None) and returned; set_short_time(out=False) switches the output off."""
        if out is False:
            check(_lib.load().corr_set_short_time(self.h, 0, None), "corr_set_short_time")
            self._st = None
            return None
        if out is None:
            out = torch.zeros((self.n_spectra // block_spectra, self.n_chan, 2, self.n_base), dtype=torch.int32,
                              device=self.device)
        check(_lib.load().corr_set_short_time(self.h, int(block_spectra), _ptr(out)), "corr_set_short_time")
        self._st = out  # keep the buffer alive while the library writes into it
        return out

    def xengine_cross(self, chan_in, p0: int, n_p: int, q0: int, n_q: int, gains=None, out=None, stream=None):
        """Cross-only rectangle V_ij, i in [p0, p0 + n_p), j in [q0, q0 + n_q), of one
        integration: [n_chan, n_p, n_q, 2] int32 (INT8) or [n_chan, n_p, n_q] complex64."""
        if out is None:
            if self.precision == "int8":
                out = torch.empty((self.n_chan, n_p, n_q, 2), dtype=torch.int32, device=self.device)
            else:
                out = torch.empty((self.n_chan, n_p, n_q), dtype=torch.complex64, device=self.device)
        check(_lib.load().corr_xengine_cross(self.h, _ptr(chan_in), _ptr(gains), int(p0), int(n_p), int(q0), int(n_q),
                                             _ptr(out), _stream(stream)), "corr_xengine_cross")
        return out

    def accum(self, out=None, stream=None):
        out = self.accum_buffer() if out is None else out
        corr_get_accum(self.h, out, stream)
        return out

    def dump(self, out=None, stream=None, copy=True):
        if copy and out is None:
            out = torch.empty((self.n_chan, self.n_base), dtype=torch.complex128, device=self.device)
        corr_dump(self.h, out if copy else None, stream)
        return out

    def flush(self, stream=None):
        """Complete a deferred dump now (see corr_dump)."""
        corr_flush(self.h, stream)

    def set_delays(self, delays=None):
        """Per-input delays in samples (sequence of n_in floats) for delay compensation
        in the F-engine, or None to switch it off."""
        if delays is None:
            check(_lib.load().corr_set_delays(self.h, None), "corr_set_delays")
            return
        d = np.ascontiguousarray(np.asarray(delays, dtype=np.float32).reshape(-1))
        if d.size != self.n_in:
            raise ValueError(f"expected {self.n_in} delays, got {d.size}")
        check(_lib.load().corr_set_delays(self.h, d.ctypes.data), "corr_set_delays")

    def check_status(self, stream=None):
        corr_check_status(self.h, stream)

    def restore_vis(self, vis=None, stream=None):
        """Checkpoint / resume: set the FP64 long integration to `vis` ([n_chan, B]
        complex128 on the device, e.g. an earlier dump()), or to zeros."""
        if vis is not None and (vis.dtype != torch.complex128 or tuple(vis.shape) != (self.n_chan, self.n_base)
                                or not vis.is_contiguous()):
            raise ValueError(f"vis must be a contiguous complex128 [{self.n_chan}, {self.n_base}] tensor")
        corr_restore_vis(self.h, vis, stream)

    def reset(self, stream=None):
        corr_reset(self.h, stream)

    def set_stage_timing(self, on: bool = True):
        """Bracket each stage's kernels with CUDA events (see stage_times)."""
        check(_lib.load().corr_set_stage_timing(self.h, 1 if on else 0), "corr_set_stage_timing")

    def stage_times(self):
        """{stage: (milliseconds, kernel launches)} since the last read (then cleared);
        waits for the recorded events."""
        n = len(_lib.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        check(_lib.load().corr_stage_times(self.h, ms, cnt), "corr_stage_times")
        return {name: (float(ms[k]), int(cnt[k])) for k, name in enumerate(_lib.STAGES)}

    def backward(self, grad_vis, chan_in, gains=None, want_chan=True, want_gains=True, stream=None):
        gc = torch.empty_like(chan_in) if want_chan else None
        gg = torch.empty(self.n_in, dtype=torch.complex64, device=self.device) if want_gains else None
        corr_backward(self.h, grad_vis, chan_in, gains, gc, gg, stream)
        return gc, gg


def corr_batch_create(subs, device: int = -1) -> ctypes.c_void_p:
    """subs: sequence of (planes, n_in, n_chan, n_spectra, vis) with device tensors."""
    arr = (_lib.corr_sub_desc * len(subs))()
    for k, (planes, n_in, n_chan, K, vis) in enumerate(subs):
        arr[k] = _lib.corr_sub_desc(int(n_in), int(n_chan), int(K), 0, _ptr(planes), _ptr(vis))
    o = corr_opts(PREC["int8"], XENG["auto"], _lib.CORR_FLAG_PLANAR, int(device))
    b = ctypes.c_void_p()
    check(_lib.load().corr_batch_create(len(subs), arr, ctypes.byref(o), ctypes.byref(b)), "corr_batch_create")
    return b


def corr_batch_tune(b, cache_path=None, stream=None) -> None:
    check(_lib.load().corr_batch_tune(b, None if cache_path is None else str(cache_path).encode(), _stream(stream)),
          "corr_batch_tune")


def corr_batch_run(b, stream=None) -> None:
    check(_lib.load().corr_batch_run(b, _stream(stream)), "corr_batch_run")


def corr_batch_check_status(b, stream=None) -> None:
    check(_lib.load().corr_batch_check_status(b, _stream(stream)), "corr_batch_check_status")


def corr_batch_channels_per_tile(b, sub: int) -> int:
    return int(_lib.load().corr_batch_channels_per_tile(b, int(sub)))


def corr_batch_destroy(b) -> None:
    check(_lib.load().corr_batch_destroy(b), "corr_batch_destroy")


class Batch:
    """Batched INT8 X-engine over sub-arrays given as planar FP16 code tensors
    [n_chan, 2, n_in, n_spectra]; allocates one INT32 output per sub-array."""

    def __init__(self, planes_list):
        self.planes = [p.contiguous() for p in planes_list]
        self.vis = []
        subs = []
        for p in self.planes:
            n_chan, two, n_in, K = p.shape
            assert two == 2 and p.dtype == torch.float16
            v = torch.zeros((n_chan, n_in * (n_in + 1) // 2, 2), dtype=torch.int32, device=p.device)
            self.vis.append(v)
            subs.append((p, n_in, n_chan, K, v))
        dev = self.planes[0].device.index if self.planes else -1
        self.b = corr_batch_create(subs, -1 if dev is None else dev)

    def tune(self, cache_path=None, stream=None):
        corr_batch_tune(self.b, cache_path, stream)

    def run(self, stream=None):
        corr_batch_run(self.b, stream)

    def check_status(self, stream=None):
        corr_batch_check_status(self.b, stream)

    def channels_per_tile(self, sub):
        return corr_batch_channels_per_tile(self.b, sub)

    def close(self):
        if getattr(self, "b", None) is not None:
            corr_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
