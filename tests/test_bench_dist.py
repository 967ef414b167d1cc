"""The multi-process logic of bench.py (replicas: the slowest rank's time
per repetition, the median repetition, the whole-job rate) on two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # per-repetition times: rank 1 is slower in the first, rank 0 in the second
    reps = bench.max_over_ranks([1.0 + rank, 3.0 - rank, 2.0], dist)
    ms = float(sorted(reps)[1])                       # the median repetition
    rate = bench.job_rate(1000, world, ms)
    out[rank] = (tuple(reps), ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert out[0] == out[1] == ((2.0, 3.0, 2.0), 2.0, pytest.approx(2 * 1000 / 2e-3))


def test_single_process_aggregation():
    import bench
    assert bench.max_over_ranks([3.5, 1.0], None) == [3.5, 1.0]
    assert bench.job_rate(10, 1, 5.0) == pytest.approx(2000.0)
