"""The N > 1 path of bench.py on CPU: two gloo ranks.  Every rank runs a
replica of the workload (no data-path collective); the job time is the
maximum over ranks and the throughput counts the work of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_seconds = [2.0, 3.5][rank]
        t = bench.max_over_ranks(local_seconds, world)
        value = bench.job_throughput(world, 1.0e12, 3, t)
        out[rank] = (t, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    t, value = out[0]
    assert t == 3.5
    assert abs(value - 2 * 3 * 1.0e12 / 3.5 / 1e12) < 1e-12


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_throughput(1, 2e12, 2, 4.0) == 1.0
