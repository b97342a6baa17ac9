"""GPU tests of the continuous-batching rollout server (mc_server_*).

The fitness a search loop reads back is the mean bead displacement after n
steps.  A rollout's result must be bitwise the same alone and in a mix with
others admitted and retired around it, and must agree with advancing the
world directly (different reduction order: within float rounding).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2607_02954_gb300 import synth
from tests.helpers import t2n

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import Server  # noqa: F401  (loads libmc)
    yield


def _specs(n=12):
    rng = np.random.default_rng(5)
    out = []
    for k in range(n):
        side = int(rng.choice([64, 128]))
        out.append((synth.world_random(100 + k, side, int(rng.integers(1, 12))), int(rng.integers(20, 61))))
    return out


def test_served_results_equal_alone_and_direct():
    from paper_2607_02954_gb300 import Server, World
    specs = _specs()
    # the mix: few slots, short ticks, so worlds join and leave while others run
    srv = Server(max_slots=5, steps_per_tick=7)
    tickets = [srv.submit(sp, n) for sp, n in specs]
    mixed = [srv.wait(t) for t in tickets]
    srv.close()
    for (sp, n), r in zip(specs, mixed):
        assert r["status"] == 0 and r["n_steps"] == n
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
        alone = Server(max_slots=1, steps_per_tick=13)
        ra = alone.wait(alone.submit(sp, n))
        alone.close()
        assert ra["com_disp"] == r["com_disp"], (ra, r)
        w = World(sp)
        w.step(n)
        direct = w.state()["disp"].astype(np.float64).mean(0)
        w.close()
        assert np.allclose(direct, r["com_disp"], rtol=1e-5, atol=1e-7)


def test_served_c4_range_and_large_worlds_equal_alone():
    """Worlds at the top of the C4 range (256^2 grids with up to 64
    filaments of up to 64 beads) and a 512^2 world, whose bins span four
    scan blocks, so the mixed plan runs the two-kernel bin scan while plans
    of the smaller worlds alone run the one-kernel scan: each rollout's
    result is bitwise the same in the mix and alone."""
    from paper_2607_02954_gb300 import Server
    rng = np.random.default_rng(17)
    specs = [(synth.world_random(300 + k, 256, int(rng.integers(32, 65))), int(rng.integers(25, 50)))
             for k in range(6)]
    specs.append((synth.world_random(399, 512, 48), 33))
    srv = Server(max_slots=4, steps_per_tick=6)
    mixed = [srv.wait(t) for t in [srv.submit(sp, n) for sp, n in specs]]
    srv.close()
    for (sp, n), r in zip(specs, mixed):
        assert r["status"] == 0 and r["n_steps"] == n
        alone = Server(max_slots=1, steps_per_tick=11)
        ra = alone.wait(alone.submit(sp, n))
        alone.close()
        assert ra["com_disp"] == r["com_disp"], (ra, r)


def test_served_result_matches_oracle_displacement():
    from paper_2607_02954_gb300 import Server
    sp = synth.world_c1(2)
    srv = Server()
    r = srv.wait(srv.submit(sp, 40))
    srv.close()
    st = O.rollout(O.World(sp), 40)
    want = t2n(st.D).mean(0)
    assert np.max(np.abs(np.array(r["com_disp"]) - want)) < 1e-5


def test_admission_respects_the_memory_budget():
    from paper_2607_02954_gb300 import Server
    specs = [(synth.world_random(200 + k, 128, 4), 30) for k in range(4)]
    # a budget below one world's footprint: only a lone world is admitted, so
    # rollouts run one after another although slots are free
    srv = Server(hbm_budget_bytes=1, max_slots=16, steps_per_tick=10)
    tickets = [srv.submit(sp, n) for sp, n in specs]
    res = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    for a, b in zip(res, res[1:]):
        assert b["t_admit_ns"] >= a["t_done_ns"]
    assert stats["submitted"] == 4 and stats["completed"] == 4


def test_poll_wait_timeout_and_unknown_tickets():
    from paper_2607_02954_gb300 import Server
    from paper_2607_02954_gb300._lib import MCError
    srv = Server(steps_per_tick=5)
    t = srv.submit(synth.world_c1(0), 3000)
    assert srv.poll(t) is None                   # still running
    with pytest.raises(MCError) as ei:
        srv.wait(t, timeout_ms=1)
    assert ei.value.status == 4                  # MC_ERR_TIMEOUT
    r = srv.wait(t)
    assert r["status"] == 0
    with pytest.raises(MCError) as ei:
        srv.poll(t)                              # collected already
    assert ei.value.status == 7
    with pytest.raises(MCError) as ei:
        srv.poll(987654321)
    assert ei.value.status == 7
    srv.close()


def test_invalid_requests_are_rejected_or_reported():
    from paper_2607_02954_gb300 import Server
    from paper_2607_02954_gb300._lib import MCError
    srv = Server()
    bad = synth.tiny_world(0, side=16, lengths=(4,))
    bad.H = 12                                   # not a multiple of 8: refused at submit
    with pytest.raises(MCError) as ei:
        srv.submit(bad, 10)
    assert ei.value.status == 1
    nan = synth.tiny_world(0, side=16, lengths=(4,))
    nan.x = nan.x.copy()
    nan.x[1] = np.nan                            # caught when the world is created
    r = srv.wait(srv.submit(nan, 10))
    assert r["status"] == 1
    # a runaway fluid trips the velocity watchdog; other rollouts are unaffected
    fast = synth.tiny_world(0, side=16, lengths=(4,))
    H, W = fast.H, fast.W
    feq = O.equilibrium(torch.ones(H, W, dtype=torch.float64), torch.full((H, W), 0.6, dtype=torch.float64),
                        torch.zeros(H, W, dtype=torch.float64))
    fast.f0 = t2n(feq - O.d2q9_weights()[:, None, None]).astype(np.float32)
    ok = synth.tiny_world(1, side=16, lengths=(4,))
    t1, t2 = srv.submit(fast, 5), srv.submit(ok, 5)
    assert srv.wait(t1)["status"] == 5
    assert srv.wait(t2)["status"] == 0
    srv.close()
