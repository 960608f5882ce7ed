"""Multi-process behaviour on CPU.

* bench.py launched with WORLD_SIZE > 1 touches no GPU: rank 0 prints one
  "unavailable" line, every rank exits 0.
* The tau-point sharding of paper_2404_17744_gb300.shard, run over two gloo
  ranks with the oracle as the per-rank evaluator and an all-gather as the
  merge, reproduces the single-process Sigma(tau) exactly.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("rank", [0, 1])
def test_bench_refuses_multi_gpu_launch(rank):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()), CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    if rank == 0:
        assert len(lines) == 1
        d = json.loads(lines[0])
        assert d["value"] is None and "unavailable" in d and d["n_gpus"] == 2
    else:
        assert lines == []


def test_tau_shards_cover_the_grid():
    from paper_2404_17744_gb300.shard import mirror_partners, tau_shard
    for n_tau in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                a, b = tau_shard(n_tau, r, world)
                got.extend(range(a, b))
                assert b - a in (n_tau // world, n_tau // world + 1)
            assert got == list(range(n_tau))
    assert mirror_partners(0, 3, 10) == [9, 8, 7]
    with pytest.raises(ValueError):
        tau_shard(4, 2, 2)


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sys.path.insert(0, ROOT)
        from oracle import thc_oracle as o
        from paper_2404_17744_gb300.shard import tau_shard
        from workloads import synth
        case = synth.make_sigma_case(8, 20, 7, 20.0, 3)
        a, b = tau_shard(case.n_tau, rank, world)
        part = o.sigma_thc(case.X, case.V, case.G_tau[a:b], case.G_bmt[a:b])
        parts = [None] * world
        dist.all_gather_object(parts, (a, part))
        merged = np.concatenate([p for _, p in sorted(parts, key=lambda x: x[0])])
        out[rank] = merged.tobytes()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_merge_tau():
    from oracle import thc_oracle as o
    from workloads import synth
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
    case = synth.make_sigma_case(8, 20, 7, 20.0, 3)
    ref = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt)
    for r in range(2):
        got = np.frombuffer(out[r], dtype=np.float64).reshape(ref.shape)
        assert np.array_equal(got, ref)
