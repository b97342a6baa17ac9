"""Host-side failure paths of the library and the rollout server, each made
on the host (no fault on the device): a full request queue, a world
allocation that fails (a fake of the allocator, armed through
mc_inject_world_alloc_failure), and cancelled requests.  In every case the
other rollouts finish with the results they give alone."""
import time

import numpy as np
import pytest
import torch

from paper_2607_02954_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_02954_gb300 import Server  # noqa: F401  (loads libmc)
    yield


def _specs(n, seed=41):
    rng = np.random.default_rng(seed)
    return [(synth.world_random(500 + k, int(rng.choice([64, 128])), int(rng.integers(1, 10))),
             int(rng.integers(20, 50))) for k in range(n)]


def _alone(spec, n):
    from paper_2607_02954_gb300 import Server
    srv = Server(max_slots=1, steps_per_tick=9)
    r = srv.wait(srv.submit(spec, n))
    srv.close()
    return r


def _wait_admitted(srv, timeout_s=30.0):
    """Bounded wait until the server's queue is empty (everything admitted)."""
    deadline = time.monotonic() + timeout_s
    while srv.stats()["pending"] > 0:
        assert time.monotonic() < deadline, "request not admitted in time"
        time.sleep(0.001)


def test_full_queue_returns_busy_and_frees_up():
    from paper_2607_02954_gb300 import Server
    from paper_2607_02954_gb300._lib import MCError
    srv = Server(max_slots=1, steps_per_tick=50, max_pending=2)
    long = srv.submit(synth.world_c1(0), 20000)   # holds the only slot
    _wait_admitted(srv)
    small = synth.tiny_world(3, side=32, lengths=(6, 5))
    a, b = srv.submit(small, 5), srv.submit(small, 6)
    with pytest.raises(MCError) as ei:
        srv.submit(small, 7)
    assert ei.value.status == 6                     # MC_ERR_BUSY: the queue holds max_pending requests
    assert srv.stats()["pending"] == 2
    assert srv.cancel(long)
    assert srv.wait(long)["status"] == 8            # MC_ERR_CANCELLED
    ra, rb = srv.wait(a), srv.wait(b)
    assert ra["status"] == 0 and rb["status"] == 0
    assert ra["com_disp"] == _alone(small, 5)["com_disp"]
    c = srv.submit(small, 7)                        # room again
    assert srv.wait(c)["status"] == 0
    srv.close()


def test_cancel_queued_and_running_rollouts():
    from paper_2607_02954_gb300 import Server
    specs = _specs(4)
    srv = Server(max_slots=3, steps_per_tick=5)
    long = srv.submit(synth.world_c1(1), 20000)
    tickets = [srv.submit(sp, n) for sp, n in specs]
    queued = srv.submit(synth.world_c1(2), 5000)
    # the last request waits behind the others (3 slots): cancel it in the queue
    assert srv.cancel(queued)
    rq = srv.wait(queued, timeout_ms=1000)
    assert rq["status"] == 8 and rq["com_disp"] == (0.0, 0.0)
    # the long rollout is running alongside the others: cancel it
    assert srv.cancel(long)
    assert srv.wait(long)["status"] == 8
    for (sp, n), t in zip(specs, tickets):
        r = srv.wait(t)
        assert r["status"] == 0
        assert r["com_disp"] == _alone(sp, n)["com_disp"]
    assert not srv.cancel(tickets[0])               # collected already
    assert not srv.cancel(123456789)                # unknown
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == stats["submitted"] == 6


def test_world_allocation_failure_reports_oom_and_spares_the_others():
    from paper_2607_02954_gb300 import Server, World, _lib
    from paper_2607_02954_gb300._lib import MCError
    lib = _lib.load()
    spec = synth.world_c1(0)
    _lib.check(lib.mc_inject_world_alloc_failure(1))
    with pytest.raises(MCError) as ei:
        World(spec)
    assert ei.value.status == 2                     # MC_ERR_OOM
    w = World(spec)                                 # the next allocation is real again
    w.step(3)
    w.check()
    w.close()
    specs = _specs(5, seed=43)
    srv = Server(max_slots=8, steps_per_tick=7)
    _lib.check(lib.mc_inject_world_alloc_failure(3))   # the third admitted world fails
    res = [srv.wait(t) for t in [srv.submit(sp, n) for sp, n in specs]]
    srv.close()
    _lib.check(lib.mc_inject_world_alloc_failure(0))
    assert res[2]["status"] == 2
    for k in (0, 1, 3, 4):
        assert res[k]["status"] == 0
        assert res[k]["com_disp"] == _alone(*specs[k])["com_disp"]


@pytest.mark.parametrize("observe", [False, True])
def test_save_and_resume_continue_the_world_bitwise(observe):
    """Checkpoint and resume: a world saved after 13 steps, destroyed, and
    loaded again continues exactly as the world that never stopped (state,
    fluid, observables, step counter)."""
    from paper_2607_02954_gb300 import World
    spec = synth.world_random(61, 128, 12)
    if observe:
        spec = synth.with_observables(spec, 61)
    a = World(spec)
    a.step(30)
    want, want_obs = a.state(fluid=True), a.observables()
    a.close()
    b = World(spec)
    b.step(13)
    image = b.save()
    b.close()
    c = World.load(image, spec)
    assert c.info()["t"] == 13
    c.step(17)
    got = c.state(fluid=True)
    for k in want:
        assert np.array_equal(want[k], got[k]), k
    assert c.observables() == want_obs
    assert c.info()["t"] == 30
    c.close()
