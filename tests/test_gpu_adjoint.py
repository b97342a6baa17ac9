"""GPU tests of the reverse mode (mc_rollout_forward / mc_rollout_backward).

The hand-written adjoint in FP32 is compared with the FP64 oracle's
reverse-mode gradient (torch.autograd through the oracle's rollout) and with
FP64 central finite differences of the oracle's loss; the gradient must not
depend on the checkpoint spacing.  Tolerance: 1e-3 of the gradient's scale.
"""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import t2n

pytestmark = pytest.mark.gpu

RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import World  # noqa: F401  (loads libmc)
    yield


def _gpu_grad(spec, n, K, gx, gy):
    from paper_2607_02954_gb300 import World
    w = World(spec)
    w.rollout_forward(n, K)
    g = w.rollout_backward(torch.as_tensor(gx, dtype=torch.float32).cuda(),
                           torch.as_tensor(gy, dtype=torch.float32).cuda())
    out = t2n(g).astype(np.float64)
    w.close()
    return out


def _oracle_grad(spec, n, gx, gy):
    ow = O.World(spec)
    return t2n(O.final_position_gradient(ow, n, torch.as_tensor(gx, dtype=torch.float64),
                                         torch.as_tensor(gy, dtype=torch.float64)))


@pytest.mark.parametrize("case", ["tiny", "c1", "custom", "red_black", "red_black_c1", "two_layer", "two_layer_c1",
                                  "direct", "direct_c1", "direct_no_passes", "direct_red_black"])
def test_adjoint_matches_oracle_reverse_mode(case):
    rng = np.random.default_rng(3)
    if case == "direct":
        spec, n, K = synth.tiny_world(5, side=32, lengths=(9, 8, 6, 2)), 30, 7
        spec.params = synth.Params(ib=1, mdf_iters=2)
    elif case == "direct_c1":
        spec, n, K = synth.world_c1(3), 20, 8
        spec.params = synth.Params(ib=1, mdf_iters=3)
    elif case == "direct_no_passes":
        spec, n, K = synth.tiny_world(6, side=32, lengths=(9, 7, 6)), 25, 6
        spec.params = synth.Params(ib=1, mdf_iters=0)
    elif case == "direct_red_black":
        spec, n, K = synth.world_random(15, 64, 4), 20, 7
        spec.params = synth.Params(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0,
                                   sigma=0.8, orient=1.0, n_pbd=3, pbd_order=1, ib=1, mdf_iters=1)
    elif case == "two_layer":
        spec, n, K = synth.tiny_world(5, side=32, lengths=(9, 8, 6, 2)), 30, 7
        spec.params = synth.Params(layers=2, layer_half=0.8)
    elif case == "two_layer_c1":
        spec, n, K = synth.world_c1(2), 20, 8
        spec.params = synth.Params(layers=2, layer_half=1.3, pbd_order=1)
    elif case == "tiny":
        spec, n, K = synth.tiny_world(3, side=32, lengths=(9, 7, 6)), 30, 7
    elif case == "red_black":
        spec, n, K = synth.tiny_world(3, side=32, lengths=(9, 8, 6, 2)), 30, 7
        spec.params = synth.Params(pbd_order=1, k_bend=0.7, k_stretch=0.6, k_shear=0.4)
    elif case == "red_black_c1":
        spec, n, K = synth.world_c1(1), 20, 8
        spec.params = synth.Params(pbd_order=1)
    elif case == "c1":
        spec, n, K = synth.world_c1(1), 20, 8
    else:
        spec, n, K = synth.world_random(9, 64, 4), 25, 10
        spec.params = synth.Params(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0,
                                   sigma=0.8, orient=1.0, n_pbd=3)
    gx = rng.standard_normal(spec.N)
    gy = rng.standard_normal(spec.N)
    g_gpu = _gpu_grad(spec, n, K, gx, gy)
    g_or = _oracle_grad(spec, n, gx, gy)
    scale = np.max(np.abs(g_or))
    assert scale > 0
    err = np.max(np.abs(g_gpu - g_or))
    assert err <= RTOL * scale, (err, scale)


def test_adjoint_independent_of_checkpoint_spacing():
    rng = np.random.default_rng(4)
    spec, n = synth.tiny_world(5, side=32, lengths=(10, 8)), 30
    gx, gy = rng.standard_normal(spec.N), rng.standard_normal(spec.N)
    gs = [_gpu_grad(spec, n, K, gx, gy) for K in (1, 10, 30)]
    scale = np.max(np.abs(gs[0]))
    for g in gs[1:]:
        assert np.max(np.abs(g - gs[0])) <= 1e-5 * scale


def test_world_continues_from_the_final_state_after_backward():
    from paper_2607_02954_gb300 import World
    spec = synth.world_c1(4)
    a, b = World(spec), World(spec)
    a.step(12)
    b.rollout_forward(12, 5)
    b.rollout_backward(torch.zeros(spec.N, device="cuda"), torch.zeros(spec.N, device="cuda"))
    sa, sb = a.state(fluid=True), b.state(fluid=True)
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    a.step(3)
    b.step(3)
    assert np.array_equal(a.state()["x"], b.state()["x"])


def _loss_worker(args):
    """The oracle's folding loss with theta0 moved by eps along direction."""
    spec, n, poly, direction, eps = args
    torch.set_num_threads(2)
    ow = O.World(spec)
    th0 = ow.theta0 if direction is None else ow.theta0 + eps * torch.as_tensor(direction)
    loss, _ = O.folding_loss(ow, n, poly, th0)
    return float(loss)


@pytest.mark.parametrize("n", [200, 2000])
def test_folding_loss_and_gradient_against_finite_differences(n):
    """Folding world (256 x 256 grid, 64 filaments x 48 beads, seeded polyline
    target) over n steps with checkpoints every 100 (n = 2000 is the folding
    workload's full length): GPU loss against the oracle's, and the GPU
    gradient's directional derivatives against FP64 central differences of
    the oracle loss along 8 random directions (eps = 1e-4; at 2000 steps the
    central differences with eps = 1e-3, 1e-4 and 1e-5 agree to 7 digits, so
    the rollout is smooth in theta0 and the differences are well
    conditioned)."""
    from paper_2607_02954_gb300 import World
    spec, poly = synth.world_c5(0)
    K, eps = 100, 1e-4
    w = World(spec)
    w.rollout_forward(n, K)
    loss, gx, gy = w.loss_polyline(poly)
    g = t2n(w.rollout_backward(gx, gy)).astype(np.float64)
    w.close()
    rng = np.random.default_rng(8)
    dirs = []
    for _ in range(8):
        d = rng.standard_normal(spec.J)
        dirs.append(d / np.linalg.norm(d))
    jobs = [(spec, n, poly, None, 0.0)]
    for d in dirs:
        jobs += [(spec, n, poly, d, eps), (spec, n, poly, d, -eps)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(8) as pool:
        losses = pool.map(_loss_worker, jobs)
    want_loss = losses[0]
    assert abs(float(loss.item()) - want_loss) <= 1e-4 * abs(want_loss)
    for k, d in enumerate(dirs):
        fd = (losses[1 + 2 * k] - losses[2 + 2 * k]) / (2 * eps)
        ad = float(np.dot(g, d))
        assert abs(ad - fd) <= RTOL * max(abs(fd), 1e-3 * np.linalg.norm(g)), (ad, fd)


@pytest.mark.parametrize("stored", [False, True])
def test_rollout_fn_autograd_bridge(stored):
    from paper_2607_02954_gb300 import World
    from paper_2607_02954_gb300.autograd import rollout_displacement
    spec = synth.tiny_world(6, side=32, lengths=(8, 8))
    th0 = torch.tensor(spec.theta0, device="cuda", requires_grad=True)
    disp = rollout_displacement(th0, spec, 15, 4, stored=stored)
    c = torch.linspace(-1, 1, disp.numel(), device="cuda").reshape(disp.shape)
    (disp * c).sum().backward()
    w = World(spec)
    w.rollout_forward(15, 4)
    direct = w.rollout_backward(c[:, 0].contiguous(), c[:, 1].contiguous())
    assert torch.allclose(th0.grad, direct, rtol=1e-5, atol=1e-7)
    w.close()


@pytest.mark.parametrize("case", ["tiny", "custom", "red_black", "two_layer", "direct"])
def test_rest_length_and_stiffness_gradients_match_oracle(case):
    """mc_rollout_backward_params: gradients with respect to theta0, every
    edge's rest length and (k_bend, k_stretch, k_shear) against the FP64
    oracle's reverse mode, 1e-3 of each gradient's scale."""
    from paper_2607_02954_gb300 import World
    rng = np.random.default_rng(11)
    if case == "tiny":
        spec, n, K = synth.tiny_world(4, side=32, lengths=(9, 7, 6)), 25, 6
    elif case == "red_black":
        spec, n, K = synth.world_random(13, 64, 5), 20, 7
        spec.params = synth.Params(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0,
                                   sigma=0.8, orient=1.0, n_pbd=3, pbd_order=1)
    elif case == "two_layer":
        spec, n, K = synth.world_random(14, 64, 5), 20, 7
        spec.params = synth.Params(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0,
                                   sigma=0.8, orient=1.0, n_pbd=3, layers=2, layer_half=0.6)
    elif case == "direct":
        spec, n, K = synth.world_random(16, 64, 5), 20, 7
        spec.params = synth.Params(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0,
                                   sigma=0.8, orient=1.0, n_pbd=3, ib=1, mdf_iters=2)
    else:
        spec, n, K = synth.world_random(12, 64, 5), 20, 7
        spec.params = synth.Params(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0,
                                   sigma=0.8, orient=1.0, n_pbd=3)
    gx = rng.standard_normal(spec.N)
    gy = rng.standard_normal(spec.N)
    w = World(spec)
    w.rollout_forward(n, K)
    g = w.rollout_backward_params(torch.as_tensor(gx, dtype=torch.float32).cuda(),
                                  torch.as_tensor(gy, dtype=torch.float32).cuda())
    w.close()
    go = O.parameter_gradient(O.World(spec), n, torch.as_tensor(gx, dtype=torch.float64),
                              torch.as_tensor(gy, dtype=torch.float64))
    for key in ("theta0", "L_rest", "k"):
        got = t2n(g[key]).astype(np.float64)
        want = t2n(go[key])
        scale = np.max(np.abs(want))
        assert scale > 0, key
        err = np.max(np.abs(got - want))
        assert err <= RTOL * scale, (key, err, scale)


@pytest.mark.parametrize("R,sigma", [(128, 1.0), (64, 2.3)])
def test_splat_loss_and_gradient_match_oracle(R, sigma):
    """mc_loss_splat on the creation positions: loss and its position
    gradient against the oracle's autograd, 1e-5."""
    from paper_2607_02954_gb300 import World
    spec, _ = synth.world_c5(1)
    target = synth.target_image(np.random.default_rng(2), R)
    w = World(spec)
    loss, gx, gy = w.loss_splat(target, sigma)
    w.close()
    X = torch.tensor(np.stack([spec.x, spec.y], 1), dtype=torch.float64, requires_grad=True)
    want = O.splat_loss(X, torch.as_tensor(target, dtype=torch.float64), spec.H, spec.W, sigma)
    (g,) = torch.autograd.grad(want, X)
    assert abs(float(loss.item()) - float(want.detach())) <= 1e-5 * float(want.detach())
    got = np.stack([t2n(gx), t2n(gy)], 1).astype(np.float64)
    assert np.max(np.abs(got - t2n(g))) <= 1e-5 * np.max(np.abs(t2n(g)))


def test_splat_folding_gradient_matches_oracle():
    """The paper's folding objective end to end: rollout, splat loss at the
    final step, reverse sweep; dL/dtheta0 against the oracle's reverse mode
    through the whole rollout, 1e-3."""
    from paper_2607_02954_gb300 import World
    spec = synth.tiny_world(9, side=64, lengths=(30, 24))
    R, sigma, n, K = 32, 1.0, 25, 8
    target = synth.target_image(np.random.default_rng(9), R)
    w = World(spec)
    w.rollout_forward(n, K)
    loss, gx, gy = w.loss_splat(target, sigma)
    g = t2n(w.rollout_backward(gx, gy)).astype(np.float64)
    w.close()
    ow = O.World(spec)
    th0 = ow.theta0.clone().requires_grad_(True)
    want, _ = O.splat_folding_loss(ow, n, target, sigma, theta0=th0)
    (go,) = torch.autograd.grad(want, th0)
    assert abs(float(loss.item()) - float(want.detach())) <= 1e-4 * float(want.detach())
    assert np.max(np.abs(g - t2n(go))) <= RTOL * np.max(np.abs(t2n(go)))


def test_rewind_and_set_rest_reproduce_fresh_worlds_bitwise():
    """An optimisation loop on one world: rewinding to the rollout's start and
    setting new rest angles gives exactly the rollout of a world created with
    those rest angles."""
    from paper_2607_02954_gb300 import World
    spec = synth.tiny_world(10, side=64, lengths=(20, 14, 9))
    n, K = 30, 8
    rng = np.random.default_rng(12)
    th_new = (spec.theta0 + 0.1 * rng.standard_normal(spec.J)).astype(np.float32)
    w = World(spec)
    w.rollout_forward(n, K)
    first = w.state(fluid=True)
    w.rollout_rewind()
    w.set_rest(theta0=th_new)
    w.rollout_forward(n, K)
    moved = w.state(fluid=True)
    w.rollout_rewind()
    w.set_rest(theta0=spec.theta0)
    w.rollout_forward(n, K)
    again = w.state(fluid=True)
    w.close()
    spec2 = synth.tiny_world(10, side=64, lengths=(20, 14, 9))
    spec2.theta0 = th_new
    ref = World(spec2)
    ref.step(n)
    want = ref.state(fluid=True)
    ref.close()
    for k in first:
        assert np.array_equal(moved[k], want[k]), k
        assert np.array_equal(again[k], first[k]), k


def test_replayed_reverse_sweep_matches_the_captured_one():
    """The second backward of the same rollout (rewind + forward) replays the
    captured sweep; the gradient equals the first one bitwise (fixed-point
    scatters) and agrees with the oracle."""
    from paper_2607_02954_gb300 import World
    spec = synth.tiny_world(11, side=32, lengths=(9, 8))
    n, K = 24, 5
    rng = np.random.default_rng(13)
    gx = torch.as_tensor(rng.standard_normal(spec.N), dtype=torch.float32).cuda()
    gy = torch.as_tensor(rng.standard_normal(spec.N), dtype=torch.float32).cuda()
    w = World(spec)
    w.rollout_forward(n, K)
    g1 = t2n(w.rollout_backward(gx, gy)).astype(np.float64)
    w.rollout_rewind()
    w.rollout_forward(n, K)
    g2 = t2n(w.rollout_backward(gx, gy)).astype(np.float64)
    w.close()
    assert np.array_equal(g1, g2)
    go = t2n(O.final_position_gradient(O.World(spec), n, torch.as_tensor(t2n(gx), dtype=torch.float64),
                                       torch.as_tensor(t2n(gy), dtype=torch.float64)))
    assert np.max(np.abs(g2 - go)) <= RTOL * np.max(np.abs(go))


@pytest.mark.parametrize("ib", [0, 1])
def test_reverse_mode_is_bitwise_repeatable(ib):
    """Two worlds with the same rollout give bitwise the same loss and
    gradients with respect to theta0, the rest lengths and the stiffnesses
    (the adjoint's scatters and sums do not depend on thread order), with
    the penalty coupling and with direct forcing."""
    import dataclasses
    from paper_2607_02954_gb300 import World
    spec, poly = synth.world_c5(2)
    if ib:
        spec.params = dataclasses.replace(spec.params, ib=1, mdf_iters=2)
    n, K = 60, 20
    outs = []
    for _ in range(2):
        w = World(spec)
        w.rollout_forward(n, K)
        loss, gx, gy = w.loss_polyline(poly)
        g = w.rollout_backward_params(gx, gy)
        outs.append((t2n(loss).copy(), {k: t2n(v).copy() for k, v in g.items()}))
        w.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in outs[0][1]:
        assert np.array_equal(outs[0][1][k], outs[1][1][k]), k


@pytest.mark.parametrize("case", ["tiny", "red_black", "two_layer", "direct"])
def test_stored_rollout_gives_the_checkpointed_gradient_bitwise(case):
    """mc_rollout_forward_stored keeps every step's record, so the backward
    re-runs nothing: the same final state as plain steps, and gradients
    bitwise equal to the checkpoint-and-recompute sweep's (the same
    intermediates reach the same adjoint kernels), also after a rewind."""
    from paper_2607_02954_gb300 import World
    rng = np.random.default_rng(21)
    spec = synth.world_random(17, 64, 5)
    params = dict(nu=0.3, kappa=0.2, k_bend=0.7, k_stretch=0.6, k_shear=0.5, k_rep=1.0, sigma=0.8, orient=1.0,
                  n_pbd=3)
    if case == "red_black":
        params["pbd_order"] = 1
    elif case == "two_layer":
        params.update(layers=2, layer_half=0.6)
    elif case == "direct":
        params.update(ib=1, mdf_iters=2)
    spec.params = synth.Params(**params)
    n, K = 23, 6
    gx = torch.as_tensor(rng.standard_normal(spec.N), dtype=torch.float32).cuda()
    gy = torch.as_tensor(rng.standard_normal(spec.N), dtype=torch.float32).cuda()
    ref = World(spec)
    ref.rollout_forward(n, K)
    g_ck = {k: t2n(v).copy() for k, v in ref.rollout_backward_params(gx, gy).items()}
    state_ck = ref.state(fluid=True)
    ref.close()
    w = World(spec)
    for rep in range(2):
        if rep:
            w.rollout_rewind()
        w.rollout_forward(n, stored=True)
        g = {k: t2n(v).copy() for k, v in w.rollout_backward_params(gx, gy).items()}
        for k in g_ck:
            assert np.array_equal(g[k], g_ck[k]), (rep, k)
        st = w.state(fluid=True)
        for k in state_ck:
            assert np.array_equal(st[k], state_ck[k]), (rep, k)
    w.close()
