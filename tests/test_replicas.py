"""Multi-rank host logic of the benchmark (replicas: one world per rank, no
data-path collective), run as two gloo ranks on the CPU: every rank sees the
slowest rank's time, the whole-job rate counts all ranks' units, and ranks
build different worlds of the same size."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2607_02954_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    ms = 10.0 + 5.0 * rank
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    spec, _ = bench.make_spec("c3_14", seed=rank)
    rate = bench.whole_job_rate(spec.N, 100, ms_max * 1e-3, ws)
    dist.barrier()
    out[rank] = (ms_max, rate, spec.N, float(spec.x[:64].sum()))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_reduce_the_slowest_time():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    slowest = 10.0 + 5.0 * (ws - 1)
    for r in range(ws):
        ms_max, rate, n, _ = res[r]
        assert ms_max == slowest
        assert rate == pytest.approx(ws * n * 100 / (slowest * 1e-3))
    assert res[0][2] == res[1][2] == 2 ** 14          # same size per rank (weak scaling)
    assert res[0][3] != res[1][3]                     # different worlds (seeded by rank)


def test_max_over_ranks_without_a_group():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(10, 4, 2.0, 1) == 20.0
