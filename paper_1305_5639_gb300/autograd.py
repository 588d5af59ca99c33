"""torch.autograd.Function over the gained X-engine (forward: corr_xengine with
gains; backward: corr_backward), for gradient-based per-input gain calibration.

Gradients follow PyTorch's complex convention (dL/dRe + j dL/dIm)."""
from __future__ import annotations

import torch


class CorrFn(torch.autograd.Function):
    """V' = CorrFn.apply(X, g, corr): X [n_chan, n_in, K] complex64 channelised
    voltages, g [n_in] complex64 gains, corr an FP32 ``Correlator`` of matching
    shape. Returns the packed gained visibilities [n_chan, B] complex64 of one
    integration, V'_ij = g_i conj(g_j) sum_a X_ia conj(X_ja)."""

    @staticmethod
    def forward(ctx, X, g, corr):
        X = X.contiguous()
        g = g.contiguous()
        corr.reset()
        corr.xengine(X, g)
        V = corr.accum()
        corr.reset()
        ctx.corr = corr
        ctx.save_for_backward(X, g)
        return V

    @staticmethod
    def backward(ctx, grad_V):
        X, g = ctx.saved_tensors
        want_x, want_g = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (want_x or want_g):
            return None, None, None
        gx, gg = ctx.corr.backward(grad_V.contiguous().to(torch.complex64), X, g, want_chan=want_x,
                                   want_gains=want_g)
        return gx, gg, None
