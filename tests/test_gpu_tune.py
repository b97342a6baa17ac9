"""GPU tests of the launch configurations and the autotuner.

Every launch configuration of a plan (per-stage kernels from a CUDA graph or
the persistent cooperative step, filaments per PBD block, one or two scan
kernels) must advance the worlds bitwise the same; the tuner's choice is one
of them, made on copies of the worlds (which do not move), and cached per
class of plan.  The persistent step's bounded barrier reports a wait that
runs out instead of hanging.
"""
import numpy as np
import pytest
import torch

from paper_2607_02954_gb300 import synth

pytestmark = pytest.mark.gpu

CONFIGS = [dict(persistent=0, pbd_warps=8, scan_kernels=0), dict(persistent=4, pbd_warps=8, scan_kernels=0),
           dict(persistent=3, pbd_warps=8, scan_kernels=0), dict(persistent=0, pbd_warps=4, scan_kernels=0),
           dict(persistent=0, pbd_warps=2, scan_kernels=2), dict(persistent=4, pbd_warps=2, scan_kernels=2),
           dict(persistent=0, pbd_warps=8, scan_kernels=0, force_kernel=1),
           dict(persistent=0, pbd_warps=4, scan_kernels=2, force_kernel=1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import _lib
    _lib.load()
    yield


def _batch(observe):
    rng = np.random.default_rng(31)
    specs = [synth.world_random(700 + k, int(rng.choice([64, 128, 256])), int(rng.integers(1, 65)))
             for k in range(10)]
    specs.append(synth.world_random(799, 512, 40))   # 4096 bins: the two-kernel scan
    if observe:
        specs = [synth.with_observables(sp, 20 + k) for k, sp in enumerate(specs)]
    return specs


def _run(specs, cfg, n):
    from paper_2607_02954_gb300 import World, set_launch_config, step_batched
    ws = [World(sp) for sp in specs]
    if cfg is not None:
        set_launch_config(ws, **cfg)
    step_batched(ws, n)
    out = [(w.state(fluid=True), w.observables(), w.info()["t"]) for w in ws]
    for w in ws:
        w.check()
        w.close()
    return out


@pytest.mark.parametrize("observe", [False, True])
def test_every_launch_config_advances_batches_bitwise_the_same(observe):
    specs = _batch(observe)
    want = _run(specs, CONFIGS[0], 37)
    for cfg in CONFIGS[1:]:
        got = _run(specs, cfg, 37)
        for (a, oa, ta), (b, ob, tb) in zip(want, got):
            assert ta == tb == 37
            assert oa == ob, cfg
            for k in a:
                assert np.array_equal(a[k], b[k]), (cfg, k)


def test_every_launch_config_advances_one_world_bitwise_the_same():
    from paper_2607_02954_gb300 import World, set_launch_config
    spec = synth.world_c1(7)
    states = []
    for cfg in CONFIGS:
        w = World(spec)
        set_launch_config([w], **cfg)
        w.step(21)
        w.check()
        states.append(w.state(fluid=True))
        w.close()
    for s in states[1:]:
        for k in states[0]:
            assert np.array_equal(states[0][k], s[k]), k


@pytest.mark.parametrize("maker", ["c2", "ragged", "tiny8", "one_tile_row", "dense"])
def test_warp_specialised_force_kernel_is_bitwise_the_same(maker):
    """The warp-specialised persistent force + LBM kernel against the
    one-tile-per-block kernel on one world: the 512^2 world (many tiles per
    block), ragged tiles, a single 8 x 8 tile and a single tile row (the
    periodic folds of an axis one tile covers), and 4 beads per cell (the
    force staging in several chunks)."""
    from paper_2607_02954_gb300 import World, set_launch_config
    if maker == "c2":
        spec = synth.world_c2(3)
    elif maker == "ragged":
        spec = synth.world_random(3, (40, 72), 6)
    elif maker == "tiny8":
        spec = synth.tiny_world(2, side=8, lengths=(3, 2))
    elif maker == "one_tile_row":
        spec = synth.world_random(5, (24, 128), 6)
    else:
        spec = synth.world_dense(256, 2 ** 18, seed=4)
    n = 3 if maker == "dense" else 19   # the dense world speeds up: a few steps stay below the watchdog
    states = []
    for fk in (0, 1):
        w = World(spec)
        set_launch_config([w], force_kernel=fk)
        w.step(n)
        w.check()
        states.append(w.state(fluid=True))
        w.close()
    for k in states[0]:
        assert np.array_equal(states[0][k], states[1][k]), k


def test_autotune_choice_is_cached_and_leaves_the_worlds_alone():
    from paper_2607_02954_gb300 import World, autotune, launch_config, step_batched
    specs = _batch(False)
    ws = [World(sp) for sp in specs]
    before = [w.state(fluid=True) for w in ws]
    cfg = autotune(ws)
    assert cfg["persistent"] in (0, 3, 4) and cfg["pbd_warps"] in (8, 4, 2) and cfg["scan_kernels"] in (0, 2)
    assert cfg["force_kernel"] in (0, 1)
    assert launch_config(ws) == cfg
    for w, b in zip(ws, before):            # measured on copies: the worlds did not move
        a = w.state(fluid=True)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        assert w.info()["t"] == 0
    step_batched(ws, 37)
    got = [w.state(fluid=True) for w in ws]
    for w in ws:
        w.close()
    want = _run(specs, CONFIGS[0], 37)
    for g, (a, _, _) in zip(got, want):
        for k in a:
            assert np.array_equal(g[k], a[k]), k
    # another batch of the same class takes the cached choice
    ws2 = [World(sp) for sp in specs]
    assert autotune(ws2) == cfg
    for w in ws2:
        w.close()


def test_persistent_barrier_wait_runs_out_and_is_reported():
    """A barrier that waits for one more block than the launch has cannot
    complete: the persistent step must give up after its time limit, end,
    and report MC_ERR_TIMEOUT through the worlds' check; the context stays
    usable and later runs are correct."""
    from paper_2607_02954_gb300 import World, _lib, set_launch_config, step_batched
    from paper_2607_02954_gb300._lib import MCError
    lib = _lib.load()
    specs = _batch(False)[:4]
    ws = [World(sp) for sp in specs]
    set_launch_config(ws, persistent=4)
    _lib.check(lib.mc_debug_barrier_test(1, 2_000_000))   # 2 ms
    try:
        step_batched(ws, 3)
        torch.cuda.synchronize()
    finally:
        _lib.check(lib.mc_debug_barrier_test(0, 1_000_000_000))
    for w in ws:
        with pytest.raises(MCError) as ei:
            w.check()
        assert ei.value.status == 4
        w.close()
    got = _run(specs, dict(persistent=4, pbd_warps=8, scan_kernels=0), 5)
    want = _run(specs, CONFIGS[0], 5)
    for (a, _, _), (b, _, _) in zip(want, got):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
