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


def test_batch_workload_full_launch_sampled(cuda_ok, tmp_path):
    """The batched workload as the bench times it: all 64 seed-0 sub-arrays on a
    16-channel window each, complex int8 sigma = 16 as planar FP16 codes, one tuned
    graph-replayed launch. Sampled parity against the oracle on every sub-array (one
    channel each): the triangle of its first 64 inputs, and 16 random pairs (i >= j)
    anywhere in it; bit-exact."""
    W = 16
    subs = synth.subarrays(seed=0)
    assert len(subs) == 64
    gen = torch.Generator(device=DEV).manual_seed(0)
    planes = []
    for d in subs:
        z = torch.randn((W, 2, d["n_in"], d["n_spectra"]), generator=gen, device=DEV) * 16.0
        planes.append(torch.clamp(torch.round(z), -127, 127).to(torch.float16).contiguous())
    b = api.Batch(planes)
    b.tune(tmp_path / "tune.json")
    b.run()
    b.run()  # a replay overwrites
    b.check_status()
    rng = np.random.default_rng(0)
    for k, (d, p, v) in enumerate(zip(subs, planes, b.vis)):
        f, n_in = k % W, d["n_in"]
        X = np.ascontiguousarray(np.transpose(p[f].cpu().numpy(), (1, 2, 0)).astype(np.int8))[None]  # [1, n_in, K, 2]
        got = v[f].cpu().numpy().astype(np.int64)
        m = min(n_in, 64)
        want = oracle.cmac(X[:, :m])[0]  # the packed triangle of the first m inputs is a prefix
        assert np.array_equal(got[: m * (m + 1) // 2], want), k
        for _ in range(16):
            i, j = sorted(rng.integers(0, n_in, 2))[::-1]
            pair = oracle.cmac(X[:, [j, i]])[0]  # packed (0,0), (1,0), (1,1): (1,0) is V_ij
            assert np.array_equal(got[i * (i + 1) // 2 + j], pair[1]), (k, i, j)
    b.close()
