"""Batched persistent X-engine (one graph-replayed launch over many uneven
sub-arrays, tuned tile shapes) against the oracle: INT8 bit-exact."""
import json

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1305_5639_gb300 import api

pytestmark = pytest.mark.gpu
DEV = "cuda"


def to_planar(X):
    return np.ascontiguousarray(np.transpose(X, (0, 3, 1, 2)).astype(np.float16))


def _subs(shapes, seed):
    data = []
    for k, (n_in, n_chan, K) in enumerate(shapes):
        X = synth.chan_int8(n_chan, n_in, K, seed=seed + k)
        data.append(X)
    return data


def test_batch_uneven_subarrays_exact_and_tuned(cuda_ok, tmp_path):
    shapes = [(20, 6, 64), (32, 5, 136), (48, 3, 256), (64, 4, 72), (100, 2, 512), (130, 2, 1032), (300, 1, 200),
              (1, 3, 8)]
    data = _subs(shapes, seed=100)
    b = api.Batch([torch.from_numpy(to_planar(X)).to(DEV) for X in data])
    b.run()
    b.check_status()
    for X, v in zip(data, b.vis):
        assert np.array_equal(v.cpu().numpy().astype(np.int64), oracle.cmac(X))
    cache = tmp_path / "tune.json"
    b.tune(cache)
    choices = [b.channels_per_tile(s) for s in range(len(shapes))]
    assert all(c in (1, 2, 4) for c in choices)
    assert all(c == 1 for (n_in, _, _), c in zip(shapes, choices) if n_in > 64)
    assert json.loads(cache.read_text())  # cache written
    for v in b.vis:
        v.zero_()
    b.run()  # re-captured with the tuned plan
    b.run()  # replay: outputs are overwritten, not accumulated
    b.check_status()
    for X, v in zip(data, b.vis):
        assert np.array_equal(v.cpu().numpy().astype(np.int64), oracle.cmac(X))
    b.close()


@pytest.mark.parametrize("cpt_n_in", [(2, 64), (4, 32), (4, 17), (2, 40)])
def test_batch_channel_packing_forced_via_cache(cuda_ok, tmp_path, cpt_n_in):
    cpt, n_in = cpt_n_in
    n_chan, K = 7, 512  # odd channel count: the last pack is partial
    X = synth.chan_int8(n_chan, n_in, K, seed=cpt * 100 + n_in)
    cache = tmp_path / "c.json"
    cache.write_text(json.dumps({f"{n_in},{K}": cpt}))
    b = api.Batch([torch.from_numpy(to_planar(X)).to(DEV)])
    b.tune(cache)
    assert b.channels_per_tile(0) == cpt
    b.run()
    b.check_status()
    assert np.array_equal(b.vis[0].cpu().numpy().astype(np.int64), oracle.cmac(X))
    b.close()


def test_batch_workload_sample_subarrays(cuda_ok):
    """Sub-array shapes drawn as in the batched workload (antennas log-uniform
    32-2048, channels from {256, 1024, 4096}, 512-4096 spectra), each on a window
    of 2 channels; exact on every sub-array."""
    shapes = [(d["n_in"], 2, d["n_spectra"]) for d in synth.subarrays(seed=0)[:12]]
    data = _subs(shapes, seed=7)
    b = api.Batch([torch.from_numpy(to_planar(X)).to(DEV) for X in data])
    b.run()
    b.check_status()
    for X, v in zip(data, b.vis):
        assert np.array_equal(v.cpu().numpy().astype(np.int64), oracle.cmac(X))
    b.close()
