"""Tensor-core adjoint (FP16 hi/lo split, tcgen05) against the oracle's closed-form
calibration gradient, on shapes with ragged row tiles (n_in not a multiple of 128),
ragged spectrum tiles (K not a multiple of 128 or 16) and contraction chunks (n_in
not a multiple of 32)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _case(n_chan, n_in, K, seed, auto_w=0.0):
    X = synth.chan_sources(n_chan, n_in, K, n_src=5, seed=seed)
    g = synth.gains(n_in, seed=seed)
    M = synth.sky_model(n_chan, n_in, 5, seed=seed)
    w = synth.weights(n_in, auto_w)
    L, dX_ref, dg_ref = oracle.loss_and_grads(X, g, M, w)
    Vp = oracle.apply_gains(oracle.cmac(X), g, n_in)
    G = (2.0 * w * (Vp / K - M) / K).astype(np.complex64)  # dL/dV' (oracle side)
    return X, g, G, dX_ref, dg_ref


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _elem(a, b):
    """Element-wise error: max |a - b| over each channel's entries (first axis),
    divided by that channel's rms of b; the largest over the channels. A wrong
    row, tile edge or channel exponent shows up here at O(1) even where it hides
    inside a global norm."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    rms = np.sqrt(np.mean(np.abs(b) ** 2, axis=1))
    return float(np.max(np.max(np.abs(a - b), axis=1) / rms))


def _elem_dg(a, b):
    """max_m |dg_m - ref_m| / rms(ref)."""
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(np.abs(b) ** 2)))


# element-wise bars: ten times the 1e-4 relative-L2 gradient bar, room for the
# extreme-value tail of up to ~5e8 entries (the calibration workload)
ELEM = 1e-3


@pytest.mark.parametrize("n_in,K,n_chan,auto_w", [(64, 64, 2, 0.0), (136, 200, 3, 1.0), (520, 264, 2, 0.0),
                                                  (8, 8, 1, 1.0)])
def test_backward_tc_matches_oracle_gradient(cuda_ok, n_in, K, n_chan, auto_w):
    X, g, G, dX_ref, dg_ref = _case(n_chan, n_in, K, seed=11, auto_w=auto_w)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    dX, dg = c.backward(torch.from_numpy(G).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
    c.check_status()
    assert _rel(dX.cpu().numpy(), dX_ref) <= 1e-4
    assert _rel(dg.cpu().numpy(), dg_ref) <= 1e-4
    assert _elem(dX.cpu().numpy(), dX_ref) <= ELEM
    assert _elem_dg(dg.cpu().numpy(), dg_ref) <= ELEM
    c.close()


@pytest.mark.parametrize("scale", [1e-12, 1e6])
def test_backward_tc_gradient_scale_invariant(cuda_ok, scale):
    """The per-channel power-of-two scaling keeps FP16 in range for any gradient
    magnitude: results scale linearly."""
    n_in, K, n_chan = 72, 48, 2
    X, g, G, dX_ref, dg_ref = _case(n_chan, n_in, K, seed=3)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    Gs = (G.astype(np.complex128) * scale).astype(np.complex64)
    dX, dg = c.backward(torch.from_numpy(Gs).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
    c.check_status()
    assert _rel(dX.cpu().numpy(), dX_ref * scale) <= 1e-4
    assert _rel(dg.cpu().numpy(), dg_ref * scale) <= 1e-4
    assert _elem(dX.cpu().numpy(), dX_ref * scale) <= ELEM
    assert _elem_dg(dg.cpu().numpy(), dg_ref * scale) <= ELEM
    c.close()


def test_backward_tc_partial_outputs(cuda_ok):
    """dX alone and dL/dg alone give the same values as both together."""
    n_in, K, n_chan = 40, 24, 2
    X, g, G, dX_ref, dg_ref = _case(n_chan, n_in, K, seed=5)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    args = (torch.from_numpy(G).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(g).to(DEV))
    dX_both, dg_both = c.backward(*args)
    dX_only, _ = c.backward(*args, want_gains=False)
    _, dg_only = c.backward(*args, want_chan=False)
    c.check_status()
    assert torch.equal(dX_only, dX_both)
    assert torch.equal(dg_only, dg_both)
    assert _rel(dX_both.cpu().numpy(), dX_ref) <= 1e-4
    assert _elem(dX_both.cpu().numpy(), dX_ref) <= ELEM
    assert _elem_dg(dg_both.cpu().numpy(), dg_ref) <= ELEM
    c.close()


def test_backward_tc_unit_gains(cuda_ok):
    n_in, K, n_chan = 48, 32, 1
    X, _, G, _, _ = _case(n_chan, n_in, K, seed=9)
    ones = np.ones(n_in, np.complex64)
    c32 = api.Correlator(n_in, 1, n_chan, K)
    ref_dX, ref_dg = c32.backward(torch.from_numpy(G).to(DEV), torch.from_numpy(X).to(DEV), torch.from_numpy(ones).to(DEV))
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    dX, dg = c.backward(torch.from_numpy(G).to(DEV), torch.from_numpy(X).to(DEV), None)
    c.check_status()
    assert _rel(dX.cpu().numpy(), ref_dX.cpu().numpy()) <= 1e-4
    assert _rel(dg.cpu().numpy(), ref_dg.cpu().numpy()) <= 1e-4
    assert _elem(dX.cpu().numpy(), ref_dX.cpu().numpy()) <= ELEM
    c.close()
    c32.close()


def test_autograd_corrfn_hilo_end_to_end(cuda_ok):
    """Forward on the hi/lo TMA X-engine and backward on the tensor-core adjoint."""
    from paper_1305_5639_gb300.autograd import CorrFn

    n_in, K, n_chan = 24, 32, 2
    X = synth.chan_sources(n_chan, n_in, K, n_src=5, seed=6)
    g = synth.gains(n_in, seed=6)
    M = synth.sky_model(n_chan, n_in, 5, seed=6)
    w = synth.weights(n_in, 0.0)
    L_ref, dX_ref, dg_ref = oracle.loss_and_grads(X, g, M, w)
    c = api.Correlator(n_in, 1, n_chan, K, precision="fp16_hilo")
    Xt = torch.from_numpy(X).to(DEV).requires_grad_(True)
    gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
    V = CorrFn.apply(Xt, gt, c)
    R = V.to(torch.complex128) / K - torch.from_numpy(M).to(DEV)
    L = torch.sum(torch.from_numpy(w).to(DEV) * (R.real ** 2 + R.imag ** 2))
    L.backward()
    assert abs(L.item() - L_ref) <= 1e-3 * abs(L_ref)
    assert _rel(gt.grad.cpu().numpy(), dg_ref) <= 1e-3
    assert _rel(Xt.grad.cpu().numpy(), dX_ref) <= 1e-3
    c.close()
