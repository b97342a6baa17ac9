"""GPU tests of the search-side observables (behaviour descriptors E_bend,
E_pos of Eqs. 5-6 and the energy collected from the energy field), with a
rest-length drive and an energy field.

Tolerance: 1e-5 of the oracle's value plus half the fixed-point quantum,
2^-25, per rounded term (each bead's energy sample, and each lane's
per-step partial sum of joints or edges, is rounded to 2^-24).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import assert_field, oracle_one_step, t2n

pytestmark = pytest.mark.gpu

QUANTUM = 2.0 ** -25


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import World  # noqa: F401  (loads libmc)
    yield


def _spec(seed, side=96, n_fil=10, **kw):
    return synth.with_observables(synth.world_random(seed, side, n_fil, **kw), seed)


def _terms(spec, n_steps):
    """Upper bound on the number of rounded terms per observable: one per
    bead (energy) or one per lane of a filament's warp (E_bend, E_pos)."""
    return (spec.N + 32 * max(spec.n_fil, 1)) * n_steps


@pytest.mark.parametrize("seed,lengths", [(21, None), (22, [300, 40, 12])])
def test_observables_match_oracle(seed, lengths):
    spec = _spec(seed, n_fil=3 if lengths else 10, lengths=lengths)
    n = 30
    from paper_2607_02954_gb300 import World
    w = World(spec)
    w.step(n)
    w.check()
    got = w.observables()
    w.close()
    want = O.observables(O.World(spec), n)
    for k in ("e_bend", "e_pos", "energy"):
        assert want[k] > 0, k
        assert abs(got[k] - want[k]) <= 1e-5 * abs(want[k]) + _terms(spec, n) * QUANTUM, (k, got[k], want[k])


def test_rest_length_drive_step_and_energy_sample_match_oracle():
    """One step with the rest-length drive: forces, velocities and the
    per-bead energy sample against the oracle."""
    spec = _spec(23)
    spec.t0 = 37
    from paper_2607_02954_gb300 import World
    _, _, st1, rec = oracle_one_step(spec)
    w = World(spec)
    w.step(1)
    assert_field("F_el", w.field("fel"), t2n(rec["F_el"]), 1e-5, floor=0.05 * 4 * 2.0 ** -23)
    assert_field("U", w.field("ubead"), t2n(rec["U"]), 1e-5)
    assert_field("e_bead", w.field("ebead"), t2n(rec["e_bead"]), 1e-5)
    w.close()


def test_observables_bitwise_alone_batched_and_served():
    from paper_2607_02954_gb300 import Server, World, step_batched
    specs = [_spec(30 + k, side=int(s), n_fil=int(f)) for k, (s, f) in enumerate([(64, 3), (128, 12), (64, 1)])]
    n = 25
    alone = []
    for sp in specs:
        w = World(sp)
        w.step(n)
        alone.append(w.observables())
        w.close()
    ws = [World(sp) for sp in specs]
    step_batched(ws, n)
    for w, a in zip(ws, alone):
        assert w.observables() == a
        w.close()
    srv = Server(max_slots=2, steps_per_tick=7)
    res = [srv.wait(srv.submit(sp, n)) for sp in specs]
    srv.close()
    for r, a in zip(res, alone):
        assert (r["e_bend"], r["e_pos"], r["energy"]) == (a["e_bend"], a["e_pos"], a["energy"])


def test_reverse_sweep_keeps_the_rollouts_observables():
    from paper_2607_02954_gb300 import World
    spec = _spec(40, side=64, n_fil=4)
    a, b = World(spec), World(spec)
    a.step(20)
    b.rollout_forward(20, 6)
    b.rollout_backward(torch.ones(spec.N, device="cuda"), torch.zeros(spec.N, device="cuda"))
    assert a.observables() == b.observables()
    a.close()
    b.close()


def test_parameter_gradients_with_rest_length_drive_match_oracle():
    """With L_rest(t) = L0 (1 + A sin(...)) the reverse mode returns the
    gradient with respect to L0."""
    from paper_2607_02954_gb300 import World
    rng = np.random.default_rng(41)
    spec = synth.with_observables(synth.tiny_world(8, side=32, lengths=(9, 7)), 8, len_amp_max=0.3)
    n, K = 20, 6
    gx, gy = rng.standard_normal(spec.N), rng.standard_normal(spec.N)
    w = World(spec)
    w.rollout_forward(n, K)
    g = w.rollout_backward_params(torch.as_tensor(gx, dtype=torch.float32).cuda(),
                                  torch.as_tensor(gy, dtype=torch.float32).cuda())
    w.close()
    go = O.parameter_gradient(O.World(spec), n, torch.as_tensor(gx), torch.as_tensor(gy))
    for key in ("theta0", "L_rest", "k"):
        got, want = t2n(g[key]).astype(np.float64), t2n(go[key])
        assert np.max(np.abs(got - want)) <= 1e-3 * np.max(np.abs(want)), key
