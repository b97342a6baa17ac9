"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: cell, bin and bin-offset indices bit-exact (computed on identical
float32 positions); per-step forces, densities and velocities within 1e-5 of
the field's largest magnitude; bead positions within 1e-4 cells after 100
steps (and after C1's full 1000).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import assert_field, crop_world, oracle_one_step, periodic_diff, t2n

pytestmark = pytest.mark.gpu

RTOL_STEP = 1e-5


def fel_floor(spec):
    """Absolute accuracy floor of the elastic force in FP32: each PBD pass
    corrects unit-length edge vectors whose float32 resolution is 2^-23, and
    the force is kappa/dt times the summed corrections.  Matters only when
    the whole world is close to rest (tiny forces)."""
    p = spec.params
    return p.kappa / p.dt * max(p.n_pbd, 1) * 2.0 ** -23


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import World  # noqa: F401  (loads libmc)
    yield


def _gpu_world(spec):
    from paper_2607_02954_gb300 import World
    return World(spec)


def _compare_one_step(spec, rtol=RTOL_STEP):
    ow, st0, st1, rec = oracle_one_step(spec)
    gw = _gpu_world(spec)
    gw.step(1)
    gw.check()
    H, W = spec.H, spec.W
    out = {}
    out["fel"] = assert_field("F_el", gw.field("fel"), t2n(rec["F_el"]), rtol, floor=fel_floor(spec))
    out["fs"] = assert_field("F_s", gw.field("fs"), t2n(rec["F_s"]), rtol)
    out["rho_s"] = assert_field("rho_s", gw.field("rho_s"), t2n(rec["rho_s"]), rtol)
    out["rho_bar"] = assert_field("rho_bar", gw.field("rho_bar"), t2n(rec["rho_bar"]), rtol)
    out["force"] = assert_field("F", gw.field("force"), t2n(rec["F"]).transpose(1, 2, 0), rtol)
    out["u"] = assert_field("u", gw.field("u"), t2n(rec["u"]).transpose(1, 2, 0), rtol)
    out["U"] = assert_field("U", gw.field("ubead"), t2n(rec["U"]), rtol)
    s = gw.state(fluid=True)
    X1 = t2n(st1.X)
    if spec.N:
        dx = periodic_diff(s["x"], X1[:, 0], W)
        dy = periodic_diff(s["y"], X1[:, 1], H)
        # returned coordinates are float32: allow their rounding (half an ulp of the box size)
        tol = float(np.spacing(np.float32(max(H, W)))) + 1e-6
        assert np.max(np.abs(dx)) < tol and np.max(np.abs(dy)) < tol
    out["theta"] = assert_field("theta", s["theta"], t2n(st1.theta), 1e-6)
    out["disp"] = assert_field("disp", s["disp"], t2n(st1.D), rtol)
    fdev_want = t2n(st1.f - O.d2q9_weights()[:, None, None])
    out["fdev"] = assert_field("fdev", s["fdev"], fdev_want, rtol)
    assert gw.info()["t"] == spec.t0 + 1
    gw.close()
    return out


# ---------------------------------------------------------------------------
# a2: cell and bin indices, bit-exact.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("maker", ["c1", "ragged", "tiny8", "edges"])
def test_cell_and_bin_indices_bit_exact(maker):
    if maker == "c1":
        spec = synth.world_c1(0)
    elif maker == "ragged":
        spec = synth.world_random(3, (40, 72), 6)   # ragged 8-cell tiles on both axes
    elif maker == "tiny8":
        spec = synth.tiny_world(2, side=8, lengths=(3, 2))
    else:
        spec = synth.world_c1(1)
        # beads on integer coordinates and just below the periodic edge
        spec.x[:8] = np.float32(np.arange(8))
        spec.x[8:12] = np.nextafter(np.float32(spec.W), np.float32(0))
        spec.y[12:16] = np.float32(0.0)
    gw = _gpu_world(spec)
    cell_w, bin_w, off_w = O.cell_and_bin(spec.x, spec.y, spec.H, spec.W, gw.info()["bin_edge"])
    assert np.array_equal(gw.field("cell"), cell_w)
    gw.step(1)
    assert np.array_equal(gw.field("bin"), bin_w)
    off = gw.field("bin_off")
    assert np.array_equal(off, off_w)
    beads = gw.field("bin_beads")
    for b in range(len(off) - 1):
        got = np.sort(beads[off[b]:off[b + 1]])
        want = np.sort(np.nonzero(bin_w == b)[0])
        assert np.array_equal(got, want), b
    gw.close()


# ---------------------------------------------------------------------------
# a1-a8: every stage of one step from identical inputs.
# ---------------------------------------------------------------------------
def test_one_step_c1():
    _compare_one_step(synth.world_c1(0))


def test_one_step_random_fluid_and_late_drive():
    spec = synth.world_c1(5)
    rng = np.random.default_rng(9)
    spec.f0 = synth.random_populations(rng, spec.H, spec.W, 2e-3)
    spec.t0 = 12345
    _compare_one_step(spec)


@pytest.mark.parametrize("case", ["tiny8", "ragged", "single_dimer", "no_filaments", "long_filament",
                                  "custom_params", "dense_rows", "red_black", "red_black_long", "two_layer",
                                  "two_layer_long", "two_layer_small"])
def test_one_step_edge_cases(case):
    rng = np.random.default_rng(1)
    if case == "tiny8":
        spec = synth.tiny_world(4, side=8, lengths=(3, 2))
    elif case == "ragged":
        spec = synth.world_random(7, (40, 72), 5)
    elif case == "single_dimer":
        spec = synth._world("dimer", 16, 24, [2], np.array([23.7, 0.6], np.float32), np.array([15.9, 0.2], np.float32),
                            np.array([0.3], np.float32), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    elif case == "no_filaments":
        spec = synth._world("fluid", 24, 16, [], np.zeros(0, np.float32), np.zeros(0, np.float32),
                            np.zeros(0, np.float32), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
        spec.f0 = synth.random_populations(rng, 24, 16, 1e-3)
    elif case == "long_filament":
        spec = synth.world_random(11, 256, 2, lengths=[1500, 40])
    elif case == "two_layer":
        spec = synth.world_random(15, 128, 20)
        spec.params = synth.Params(layers=2, layer_half=0.8)
    elif case == "two_layer_long":
        spec = synth.world_random(16, 256, 3, lengths=[900, 50, 2])
        spec.params = synth.Params(layers=2, layer_half=1.7, pbd_order=1)
    elif case == "two_layer_small":
        spec = synth.tiny_world(17, side=16, lengths=(7, 5))
        spec.params = synth.Params(layers=2, layer_half=2.0)
    elif case == "red_black":
        spec = synth.world_random(13, 128, 24)
        spec.params = synth.Params(k_bend=0.8, k_stretch=0.7, k_shear=0.5, pbd_order=1, n_pbd=5)
    elif case == "red_black_long":
        spec = synth.world_random(14, 256, 3, lengths=[700, 65, 33])
        spec.params = synth.Params(pbd_order=1)
    elif case == "custom_params":
        spec = synth.world_c1(2)
        spec.params = synth.Params(nu=0.5, Lambda=3.0 / 16.0, kappa=0.2, k_bend=0.8, k_stretch=0.9,
                                   k_shear=0.6, k_rep=1.5, sigma=1.7, orient=0.0, n_pbd=7)
    else:
        spec = synth.world_rows(256, 4096, seed=3)
    _compare_one_step(spec)


@pytest.mark.parametrize("n_beads", [2 ** 18, 2 ** 19])
def test_one_step_above_one_bead_per_cell(n_beads):
    """The shape of the paper's scalability runs (a 256^2 grid with up to
    500k particles): 4 and 8 beads per cell.  A 32 x 32 tile then holds 4k
    to 8k beads, so the force kernel stages its records in several chunks,
    and the deposit's fixed-point scale comes from bins of 256 to 512
    beads."""
    _compare_one_step(synth.world_dense(256, n_beads, seed=4))


def test_one_step_c2_full_size():
    """512 x 512 grid with 262,144 beads: the whole step against the oracle."""
    _compare_one_step(synth.world_c2(0))


def _full_size_samples(spec, rng, n_random=20):
    """Random beads plus beads at the periodic seams and on tile corners."""
    picks = list(rng.choice(spec.N, n_random, replace=False))
    picks += [int(np.argmin(spec.x)), int(np.argmax(spec.x)), int(np.argmin(spec.y)), int(np.argmax(spec.y))]
    corner = (np.mod(spec.x, 32.0) < 1.0) & (np.mod(spec.y, 32.0) < 1.0)
    if corner.any():
        picks += list(rng.choice(np.nonzero(corner)[0], min(4, int(corner.sum())), replace=False))
    return picks


def test_full_size_2_22_sampled():
    """The benchmark's workload, 2^22 beads as 64-bead filaments on a 4096^2
    grid, in the launch configuration the benchmark times (CUDA-graph replay
    through mc_step).  After one step: for ~28 sampled beads, F_el, F_s, U,
    the new position and the force and velocity on the 5x5 cells around the
    bead against one oracle step of the sub-world around it (exact for those
    values).  After 16 more steps of graph replay: the world equals one
    advanced by direct launches bitwise, sum F_el = 0, sum F_s = 0,
    sum F = sum (F_el + F_s), and the populations keep the mass."""
    spec = synth.world_c3(22, 0)
    H, W = spec.H, spec.W
    gw = _gpu_world(spec)
    gw.step(1)
    gw.check()
    fel, fs, ub = gw.field("fel"), gw.field("fs"), gw.field("ubead")
    Fg, ug = gw.field("force"), gw.field("u")
    st = gw.state()
    rng = np.random.default_rng(22)
    got = {k: [] for k in ("F_el", "F_s", "U", "X", "F", "u")}
    want = {k: [] for k in got}
    for i in _full_size_samples(spec, rng):
        sub, beads, (sx, sy) = crop_world(spec, spec.x[i], spec.y[i])
        _, _, st1, rec = oracle_one_step(sub)
        k = int(np.nonzero(beads == i)[0][0])
        got["F_el"].append(fel[i]); want["F_el"].append(t2n(rec["F_el"])[k])
        got["F_s"].append(fs[i]); want["F_s"].append(t2n(rec["F_s"])[k])
        got["U"].append(ub[i]); want["U"].append(t2n(rec["U"])[k])
        X1 = t2n(st1.X)[k] + np.array([sx, sy], np.float64)
        got["X"].append(np.array([periodic_diff(st["x"][i], X1[0], W), periodic_diff(st["y"][i], X1[1], H)]))
        want["X"].append(np.zeros(2))
        cx, cy = int(np.floor(spec.x[i])), int(np.floor(spec.y[i]))
        for gy in range(cy - 2, cy + 3):
            for gx in range(cx - 2, cx + 3):
                got["F"].append(Fg[gy % H, gx % W]); want["F"].append(t2n(rec["F"])[:, (gy - sy) % sub.H, (gx - sx) % sub.W])
                got["u"].append(ug[gy % H, gx % W]); want["u"].append(t2n(rec["u"])[:, (gy - sy) % sub.H, (gx - sx) % sub.W])
    assert_field("F_el", np.array(got["F_el"]), np.array(want["F_el"]), RTOL_STEP, floor=fel_floor(spec))
    for k in ("F_s", "U", "F", "u"):
        assert_field(k, np.array(got[k]), np.array(want[k]), RTOL_STEP)
    assert np.max(np.abs(np.array(got["X"]))) <= 0.5 * np.spacing(np.float32(W))
    # whole-world properties of the same step
    tot = lambda a: np.abs(np.asarray(a, np.float64)).sum(axis=tuple(range(a.ndim - 1)))
    assert np.all(np.abs(fel.astype(np.float64).sum(0)) <= 1e-6 * tot(fel))
    assert np.all(np.abs(fs.astype(np.float64).sum(0)) <= 1e-6 * tot(fs))
    ftot = fel.astype(np.float64) + fs
    assert np.all(np.abs(Fg.astype(np.float64).sum((0, 1)) - ftot.sum(0)) <= 1e-5 * tot(ftot))
    del Fg, ug
    # 16 steps of graph replay against 16 direct steps, bitwise
    gd = _gpu_world(spec)
    gd.step(1)
    for _ in range(16):
        gd.step(1)
    gw.step(16)
    a, b = gw.state_device(), gd.state_device()
    for k in a:
        assert torch.equal(a[k], b[k]), k
    f = gw.state(fluid=True)["fdev"]
    assert abs(float(f.astype(np.float64).sum())) <= 1e-6 * H * W
    gw.close()
    gd.close()


# ---------------------------------------------------------------------------
# 100-step rollout (positions within 1e-4 cells).
# ---------------------------------------------------------------------------
def test_rollout_100_steps_c1():
    spec = synth.world_c1(0)
    ow = O.World(spec)
    st = O.rollout(ow, 100)
    gw = _gpu_world(spec)
    gw.step(100)
    gw.check()
    s = gw.state()
    X = t2n(st.X)
    err = max(np.max(np.abs(periodic_diff(s["x"], X[:, 0], spec.W))),
              np.max(np.abs(periodic_diff(s["y"], X[:, 1], spec.H))))
    assert err < 1e-4, err
    assert np.max(np.abs(s["disp"] - t2n(st.D))) < 1e-4
    assert gw.info()["t"] == 100
    gw.close()


@pytest.mark.parametrize("variant", ["red_black", "two_layer", "two_layer_red_black"])
def test_rollout_100_steps_variants(variant):
    """C1 worlds with the red-black PBD order and with two-layer filaments:
    positions and displacements after 100 steps within 1e-4 cells."""
    spec = synth.world_c1(3)
    spec.params = {"red_black": synth.Params(pbd_order=1),
                   "two_layer": synth.Params(layers=2, layer_half=0.8),
                   "two_layer_red_black": synth.Params(layers=2, layer_half=1.2, pbd_order=1)}[variant]
    st = O.rollout(O.World(spec), 100)
    gw = _gpu_world(spec)
    gw.step(100)
    gw.check()
    s = gw.state()
    X = t2n(st.X)
    err = max(np.max(np.abs(periodic_diff(s["x"], X[:, 0], spec.W))),
              np.max(np.abs(periodic_diff(s["y"], X[:, 1], spec.H))))
    assert err < 1e-4, err
    assert np.max(np.abs(s["disp"] - t2n(st.D))) < 1e-4
    gw.close()


def test_rollout_100_steps_c2():
    """The C2 world (262,144 beads on 512^2, one bead per cell) after 100
    steps: positions and displacements within 1e-4 cells of the FP64 oracle."""
    spec = synth.world_c2(0)
    st = O.rollout(O.World(spec), 100)
    gw = _gpu_world(spec)
    gw.step(100)
    gw.check()
    s = gw.state()
    X = t2n(st.X)
    err = max(np.max(np.abs(periodic_diff(s["x"], X[:, 0], spec.W))),
              np.max(np.abs(periodic_diff(s["y"], X[:, 1], spec.H))))
    assert err < 1e-4, err
    assert np.max(np.abs(s["disp"] - t2n(st.D))) < 1e-4
    gw.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_rollout_1000_steps_c1(seed):
    """The C1 configuration at its full length: positions and displacements
    after 1000 steps within 1e-4 cells of the FP64 oracle (measured: under
    5e-5; the FP32 error grows slowly, about linearly in the step count)."""
    spec = synth.world_c1(seed)
    st = O.rollout(O.World(spec), 1000)
    gw = _gpu_world(spec)
    gw.step(1000)
    gw.check()
    s = gw.state()
    X = t2n(st.X)
    err = max(np.max(np.abs(periodic_diff(s["x"], X[:, 0], spec.W))),
              np.max(np.abs(periodic_diff(s["y"], X[:, 1], spec.H))))
    assert err < 1e-4, err
    assert np.max(np.abs(s["disp"] - t2n(st.D))) < 1e-4
    gw.close()


# ---------------------------------------------------------------------------
# Batched and alone give bitwise identical worlds.
# ---------------------------------------------------------------------------
def test_batched_equals_alone_bitwise():
    from paper_2607_02954_gb300 import step_batched
    # the C4 range (sides 64..256, up to 64 filaments) plus a 512^2 world,
    # whose 4096 bins span four scan blocks (the plan runs both scan kernels)
    specs = [synth.world_random(s, side, nf) for s, side, nf in
             [(1, 64, 3), (2, 128, 17), (3, 64, 1), (4, 256, 40), (5, 128, 8), (6, 256, 64), (7, 512, 30)]]
    specs[2].params = synth.Params(pbd_order=1, sigma=0.6)   # a red-black world with a narrower filter
    specs[3].params = synth.Params(layers=2, layer_half=0.9)  # a two-layer world
    alone = []
    for sp in specs:
        w = _gpu_world(sp)
        w.step(37)
        alone.append(w.state(fluid=True))
        w.close()
    ws = [_gpu_world(sp) for sp in specs]
    step_batched(ws, 20)
    step_batched(ws, 17)
    for w, a in zip(ws, alone):
        b = w.state(fluid=True)
        for k in a:
            assert np.array_equal(a[k], b[k]), k
        assert w.info()["t"] == 37
        w.close()


def _edge_reach_world():
    """64^2 world whose tile x in [32, 64) is reached by one bead only, with
    a kernel weight too small for the deposit's fixed point: a 48-bead snake
    fills one 8 x 8 bin left of the tile edge (its count sets the deposit
    scale to 2^24, and no snake bead reaches column 32), and a stretched
    2-bead filament has its first bead at x = 30.0002, whose stencil reaches
    column 32 with weight phi(1.9998) ~ 1.5e-8 in float32."""
    xs, ys = [], []
    for r in range(8):
        row = [24.3 + k for k in range(6)]
        xs += row if r % 2 == 0 else row[::-1]
        ys += [0.5 + r] * 6
    xs += [30.0002, 28.5002]
    ys += [12.5, 12.5]
    x, y = np.array(xs, np.float32), np.array(ys, np.float32)
    d = np.stack([np.diff(x[:48]), np.diff(y[:48])], 1)
    th_snake = np.arctan2(d[:, 1], d[:, 0])
    theta = np.concatenate([th_snake, [np.pi]]).astype(np.float32)
    theta0 = np.diff(th_snake)   # the snake's rest shape is its start shape
    z = np.zeros(len(theta0))
    return synth._world("edge_reach", 64, 64, [48, 2], x, y, theta, theta0, z, z, z)


def test_batched_tile_skip_is_exact():
    """The batched force pass skips tiles that no bead's stencil reaches.  A
    tile reached only by a weight that the deposit's fixed point rounds to 0
    must still get its (tiny) spread: the world stepped alone (which never
    skips) and in a batch stay bitwise equal."""
    from paper_2607_02954_gb300 import step_batched
    spec = _edge_reach_world()
    probe = _gpu_world(spec)
    probe.step(1)
    rho, F = probe.field("rho_s"), probe.field("force")
    # the case this test is about: nothing deposited on column 32, a spread there
    assert np.all(rho[8:18, 32] == 0.0)
    assert np.any(F[8:18, 32] != 0.0)
    probe.close()
    alone = _gpu_world(spec)
    alone.step(6)
    want = alone.state(fluid=True)
    alone.close()
    ws = [_gpu_world(spec), _gpu_world(synth.world_random(3, 64, 4))]
    step_batched(ws, 6)
    got = ws[0].state(fluid=True)
    for k in want:
        assert np.array_equal(want[k], got[k]), k
    for w in ws:
        w.close()


@pytest.mark.parametrize("side,layers", [(128, 1), (40, 1), (24, 1), (64, 2)])
def test_stage_sequences_equal_the_step_bitwise(side, layers):
    """mc_step runs the fused spread + LBM kernel (stage 7); stages 0..6 run
    the same step with F through device memory (stages 4 and 5).  Both, and
    the fused stage sequence 0, 1, 2, 3, 7, 6, give the same world bitwise."""
    import ctypes
    from paper_2607_02954_gb300 import _lib
    lib = _lib.load()
    spec = synth.world_random(7, side, 6 if side < 64 else 20)
    spec.params = synth.Params(layers=layers, layer_half=1.1)
    sh = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    worlds = [_gpu_world(spec) for _ in range(3)]
    for _ in range(5):
        worlds[0].step(1)
        for sid in (0, 1, 2, 3, 4, 5, 6):
            _lib.check(lib.mc_step_stage(worlds[1].handle, sid, sh))
        for sid in (0, 1, 2, 3, 7, 6):
            _lib.check(lib.mc_step_stage(worlds[2].handle, sid, sh))
    torch.cuda.synchronize()
    st = [w.state(fluid=True) for w in worlds]
    for k in st[0]:
        assert np.array_equal(st[0][k], st[1][k]), k
        assert np.array_equal(st[0][k], st[2][k]), k
    for w in worlds:
        assert w.info()["t"] == 5
        w.close()


def test_graph_replay_equals_direct_steps_bitwise():
    spec = synth.world_c1(3)
    a = _gpu_world(spec)
    for _ in range(20):
        a.step(1)            # direct launches
    b = _gpu_world(spec)
    b.step(20)               # one 16-step graph replay + 4 direct steps
    sa, sb = a.state(fluid=True), b.state(fluid=True)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    a.close()
    b.close()


@pytest.mark.parametrize("feature", ["observables", "observables_long_filaments", "two_layers"])
def test_fused_steps_equal_single_steps_bitwise(feature):
    """A run of n >= 2 steps runs each step's PBD fused with the previous
    step's advance (16-step graph replays, then direct launches); single
    steps run them as separate kernels.  Worlds with the extended features
    (rest-length drive, energy field and observables; filaments longer than
    64 beads; two layers) give the same state, per-bead energy samples and
    observables bitwise both ways."""
    if feature == "two_layers":
        spec = synth.world_random(11, 64, 8)
        spec.params = synth.Params(layers=2, layer_half=1.1)
    elif feature == "observables_long_filaments":
        spec = synth.with_observables(synth.world_random(12, 96, 3, lengths=[300, 40, 12]), 12)
    else:
        spec = synth.with_observables(synth.world_random(13, 96, 10), 13)
    a, b = _gpu_world(spec), _gpu_world(spec)
    for _ in range(21):
        a.step(1)
    b.step(21)
    sa, sb = a.state(fluid=True), b.state(fluid=True)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    assert a.observables() == b.observables()
    if feature != "two_layers":
        assert a.observables()["energy"] > 0
        assert np.array_equal(a.field("ebead"), b.field("ebead"))
    assert a.info()["t"] == b.info()["t"] == 21
    a.close()
    b.close()


def test_device_inputs_equal_host_inputs():
    from paper_2607_02954_gb300 import World
    spec = synth.world_c1(6)
    a, b = World(spec), World(spec, device=True)
    a.step(5)
    b.step(5)
    sa, sb = a.state(fluid=True), b.state(fluid=True)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def test_watchdog_flags_runaway_velocity():
    """A fluid moving faster than the watchdog limit is reported, and the
    world's other results stay finite; a calm world passes."""
    spec = synth.tiny_world(0, side=16, lengths=(4,))
    H, W = spec.H, spec.W
    feq = O.equilibrium(torch.ones(H, W, dtype=torch.float64), torch.full((H, W), 0.6, dtype=torch.float64),
                        torch.zeros(H, W, dtype=torch.float64))
    spec.f0 = t2n(feq - O.d2q9_weights()[:, None, None]).astype(np.float32)
    from paper_2607_02954_gb300._lib import MCError
    w = _gpu_world(spec)
    w.step(1)
    with pytest.raises(MCError) as ei:
        w.check()
    assert ei.value.status == 5
    w.clear_flags()
    calm = _gpu_world(synth.tiny_world(0, side=16, lengths=(4,)))
    calm.step(3)
    calm.check()
