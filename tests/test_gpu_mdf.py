"""Direct forcing with multi-direct-forcing passes (ib = 1) on the GPU,
through the C ABI, against the FP64 oracle.

- one step from identical inputs: every field within 1e-5 of its largest
  magnitude (the parity test's comparison), for one and four passes, on a
  world at rest, a world in a random fluid and a tiny world;
- bead positions within 1e-4 cells after 100 steps;
- a batch mixing direct-forcing and penalty worlds equals each world alone,
  bitwise;
- the reverse mode and the per-stage entry refuse direct-forcing worlds.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import periodic_diff, t2n

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import World  # noqa: F401  (loads libmc)
    yield


def _world(spec):
    from paper_2607_02954_gb300 import World
    return World(spec)


def _mdf(spec, m):
    p = spec.params
    spec.params = synth.Params(**{**p.__dict__, "ib": 1, "mdf_iters": m})
    return spec


@pytest.mark.parametrize("case,m", [("c1", 1), ("c1", 4), ("fluid", 4), ("tiny", 3), ("long", 2), ("dense", 3),
                                    ("ragged", 2)])
def test_mdf_one_step_matches_oracle(case, m):
    """("dense": 2560 beads on 64^2, so more beads reach a tile than one
    staging pass holds, and the pass kernel evaluates dF twice; "ragged":
    a 40 x 72 grid, whose last tile column and row are partial.)"""
    from tests.test_gpu_parity import _compare_one_step
    if case == "c1":
        spec = synth.world_c1(2)
    elif case == "fluid":
        spec = synth.world_c1(5)
        spec.f0 = synth.random_populations(np.random.default_rng(4), spec.H, spec.W, 2e-3)
    elif case == "tiny":
        spec = synth.tiny_world(3, side=16, lengths=(6, 5, 3))
    elif case == "long":
        spec = synth.world_random(6, 64, 3, lengths=[80, 70, 12])   # filaments beyond 64 beads
    elif case == "dense":
        spec = synth.world_random(8, 64, 40, lengths=[64] * 40)
    else:
        spec = synth.world_random(9, (40, 72), 6)
    _compare_one_step(_mdf(spec, m))


def test_mdf_rollout_100_steps():
    spec = _mdf(synth.world_c1(0), 4)
    st = O.rollout(O.World(spec), 100)
    gw = _world(spec)
    gw.step(100)
    gw.check()
    s = gw.state()
    X = t2n(st.X)
    err = max(np.max(np.abs(periodic_diff(s["x"], X[:, 0], spec.W))),
              np.max(np.abs(periodic_diff(s["y"], X[:, 1], spec.H))))
    assert err < 1e-4, err
    assert np.max(np.abs(s["disp"] - t2n(st.D))) < 1e-4
    gw.close()


def test_mdf_batched_with_penalty_worlds_equals_alone_bitwise():
    from paper_2607_02954_gb300 import step_batched
    specs = [_mdf(synth.world_random(1, 64, 3), 4), synth.world_random(2, 128, 12),
             _mdf(synth.world_random(3, 128, 8), 2), synth.world_random(4, 64, 5)]
    alone = []
    for sp in specs:
        w = _world(sp)
        w.step(21)
        alone.append(w.state(fluid=True))
        w.close()
    ws = [_world(sp) for sp in specs]
    step_batched(ws, 21)
    for w, a in zip(ws, alone):
        b = w.state(fluid=True)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        w.close()


def test_mdf_worlds_refuse_stages_and_reverse_mode_ends_in_the_final_state():
    """Single stages are refused for direct-forcing worlds; a rollout with
    its reverse sweep leaves the world bitwise where plain steps take it."""
    from paper_2607_02954_gb300 import _lib
    lib = _lib.load()
    spec = _mdf(synth.tiny_world(1), 2)
    w = _world(spec)
    sh = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mc_step_stage(w.handle, 0, sh) != 0
    w.rollout_forward(8, 4)
    z = torch.ones(spec.N, dtype=torch.float32, device="cuda")
    g = w.rollout_backward(z, z)
    assert bool(torch.isfinite(g).all())
    ref = _world(spec)
    ref.step(8)
    a, b = w.state(fluid=True), ref.state(fluid=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    w.close()
    ref.close()


def test_mdf_served_mix_equals_alone_bitwise():
    """Direct-forcing requests served among penalty requests (worlds joining
    and leaving the batch) give the same result as served alone."""
    from paper_2607_02954_gb300 import Server
    specs = [(_mdf(synth.world_random(40 + k, 64, 3 + k), 2 + k % 3), 25 + 5 * k) if k % 2 == 0
             else (synth.world_random(40 + k, 64, 4), 30) for k in range(6)]
    srv = Server(max_slots=3, steps_per_tick=6)
    mixed = [srv.wait(t) for t in [srv.submit(sp, n) for sp, n in specs]]
    srv.close()
    for (sp, n), r in zip(specs, mixed):
        assert r["status"] == 0 and r["n_steps"] == n
        alone = Server(max_slots=1, steps_per_tick=11)
        ra = alone.wait(alone.submit(sp, n))
        alone.close()
        assert ra["com_disp"] == r["com_disp"], (ra, r)


@pytest.mark.parametrize("variant", ["red_black", "observables"])
def test_mdf_with_other_features_matches_oracle(variant):
    """Direct forcing with red-black PBD, and with a rest-length drive,
    energy field and observables: one step against the oracle, and the
    observables after 20 steps."""
    from tests.test_gpu_parity import _compare_one_step
    spec = synth.world_c1(7)
    if variant == "red_black":
        spec.params = synth.Params(pbd_order=1, ib=1, mdf_iters=3)
        _compare_one_step(spec)
        return
    spec.params = synth.Params(ib=1, mdf_iters=3)
    synth.with_observables(spec, 3)
    _compare_one_step(spec)
    want = O.observables(O.World(spec), 20)
    w = _world(spec)
    w.step(20)
    got = w.observables()
    w.close()
    for k in ("e_bend", "e_pos", "energy"):
        assert abs(got[k] - want[k]) <= 1e-5 * max(abs(want[k]), 1.0), (k, got[k], want[k])
