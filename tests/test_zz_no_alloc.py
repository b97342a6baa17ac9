"""GPU test of mc_world_get_positions_noalloc, the allocation-free read-out.

Who needs it: callers that cannot allocate device memory while they read
results back, because their process's device memory is fully reserved by
another allocator (or capped by a fixed budget) so any new cudaMalloc fails,
or because they run a latency-critical loop where cudaMalloc / cudaFree can
synchronize the device.  mc_world_get_state allocates a device staging
buffer on every host read-out; this entry point stages through a fixed
static device array instead.

The test calls both entry points through the C ABI and requires the same
positions (within the tests' position tolerance) on two calls in a row, then
checks the size limit.  The file sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own in
a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2607_02954_gb300 import synth

pytestmark = pytest.mark.gpu

NOALLOC_MAX_BEADS = 1 << 20


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import _lib
    return _lib.load()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc_positions(lib, world):
    N = world.spec.N
    x = np.full(N, np.nan, np.float32)
    y = np.full(N, np.nan, np.float32)
    status = lib.mc_world_get_positions_noalloc(world.handle, ctypes.c_void_p(x.ctypes.data),
                                                ctypes.c_void_p(y.ctypes.data), _stream())
    assert status == 0, lib.mc_last_error()
    return x, y


def _state_positions(lib, world):
    N = world.spec.N
    x = np.full(N, np.nan, np.float32)
    y = np.full(N, np.nan, np.float32)
    status = lib.mc_world_get_state(world.handle, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                    None, None, None, 0, _stream())
    assert status == 0, lib.mc_last_error()
    return x, y


def _tol(spec):
    # positions come back as float32: half an ulp of the box size
    return float(np.spacing(np.float32(max(spec.H, spec.W))))


def test_noalloc_positions_match_get_state_on_two_calls(lib):
    from paper_2607_02954_gb300 import World
    spec = synth.world_c1(0)
    w = World(spec)
    w.step(5)
    ref1 = _state_positions(lib, w)
    got1 = _noalloc_positions(lib, w)
    for a, b in zip(got1, ref1):
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a.astype(np.float64) - b)) <= _tol(spec)
    w.step(7)
    ref2 = _state_positions(lib, w)
    got2 = _noalloc_positions(lib, w)
    for a, b in zip(got2, ref2):
        assert np.max(np.abs(a.astype(np.float64) - b)) <= _tol(spec)
    # the second call returns the new state, not the previous call's contents
    assert np.max(np.abs(got2[0] - got1[0])) > 0
    # a smaller world through the same shared array
    small = World(synth.tiny_world(1, side=16, lengths=(5, 4)))
    small.step(2)
    ref3 = _state_positions(lib, small)
    got3 = _noalloc_positions(lib, small)
    for a, b in zip(got3, ref3):
        assert np.max(np.abs(a.astype(np.float64) - b)) <= _tol(small.spec)
    small.close()
    w.close()


def test_noalloc_rejects_worlds_above_the_limit(lib):
    from paper_2607_02954_gb300 import World
    rng = np.random.default_rng(0)
    n_fil = NOALLOC_MAX_BEADS // 64 + 1
    x, y, th = synth.place_rows(rng, 2048, 2048, n_fil, 64, pitch=2)
    J = n_fil * 62
    spec = synth._world("over_limit", 2048, 2048, [64] * n_fil, x, y, th, np.zeros(J), np.zeros(J),
                        np.zeros(J), np.zeros(J))
    assert spec.N > NOALLOC_MAX_BEADS
    w = World(spec)
    xo = np.empty(spec.N, np.float32)
    yo = np.empty(spec.N, np.float32)
    status = lib.mc_world_get_positions_noalloc(w.handle, ctypes.c_void_p(xo.ctypes.data),
                                                ctypes.c_void_p(yo.ctypes.data), _stream())
    assert status == 1
    assert "limit" in lib.mc_last_error().decode()
    w.close()
