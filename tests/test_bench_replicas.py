"""The multi-rank path of bench.py on CPU with gloo (world size 2): the path
does not shard within a model, so every rank solves its own seeded replica;
the job's time is the slowest rank's and its rate counts every rank's
updates."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 10.0 * (rank + 1)
        ms = bench.max_over_ranks(local, world, "cpu")
        models, T = bench.models_for(1, seed=rank)
        m = models[0]
        out.put((rank, ms, T, float(np.asarray(m.unary, np.float64).sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]  # both ranks see the slowest rank's time
    assert res[0][2] == res[1][2]  # the same workload ...
    assert res[0][3] != res[1][3]  # ... drawn from each rank's own seed
    # whole-job rate: both ranks' updates over the slowest rank's time
    assert bench.whole_job_rate(1000.0, world, 20.0) == pytest.approx(2000.0 / 0.020)
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
