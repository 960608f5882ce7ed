"""Batched evaluation (include/thc_batch.h): every molecule of a batch of
uneven sizes against the FP64 oracle (1e-10 for FP64, 1e-6 for 3 x BF16) and
against single-context evaluation; CUDA-graph replay; autotuner table."""
import os

import numpy as np
import pytest

from oracle import thc_oracle as o
from workloads import batch as wb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run_batch(cases, precision, tune, n_streams=3, calls=2):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    X = [torch.from_numpy(c.X).to(dev) for c in cases]
    V = [torch.from_numpy(c.V).to(dev) for c in cases]
    G = [torch.from_numpy(c.G_tau).to(dev) for c in cases]
    S = [torch.empty_like(g) for g in G]
    c0 = cases[0]
    b = thc.thc_batch_init([c.n for c in cases], [c.N for c in cases], c0.n_tau, c0.beta, X, V, c0.tau,
                           precision, n_streams, 0, tune, torch.cuda.current_stream(dev).cuda_stream)
    try:
        outs = []
        for _ in range(calls):
            for s in S:
                s.zero_()
            thc.thc_batch_eval(b, G, S)
            torch.cuda.synchronize()
            outs.append([s.cpu().numpy() for s in S])
        info = thc.thc_batch_graph_info(b)
        flops = thc.thc_batch_flops(b)
    finally:
        thc.thc_batch_destroy(b)
    return outs, info, flops


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_batch_matches_oracle_and_replays(precision, tol):
    cases = wb.make_batch(5, 1, 40, 6, 30.0, seed=7)
    cases[0] = wb.synth.make_sigma_case(1, 5, 6, 30.0, 99, n_occ=1)     # a one-orbital molecule
    outs, (kernels, nodes), flops = _run_batch(cases, precision, tune=(precision == 1))
    assert kernels > 0 and nodes >= kernels and flops > 0
    for i, c in enumerate(cases):
        ref = o.sigma_thc(c.X, c.V, c.G_tau, c.G_bmt)
        assert np.abs(outs[0][i] - ref).max() <= tol, i
        assert np.abs(outs[1][i] - outs[0][i]).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_batch_equals_single_contexts():
    from paper_2404_17744_gb300 import thc
    cases = wb.make_batch(4, 20, 70, 4, 30.0, seed=8)
    outs, _, _ = _run_batch(cases, 1, tune=False, calls=1)
    dev = torch.device("cuda:0")
    for i, c in enumerate(cases):
        ctx = thc.thc_sigma_init(c.n, c.N, c.n_tau, c.beta, torch.from_numpy(c.X).to(dev),
                                 torch.from_numpy(c.V).to(dev), c.tau, thc.THC_BF16X3, 3)
        try:
            G = torch.from_numpy(c.G_tau).to(dev)
            S = torch.empty_like(G)
            thc.thc_sigma_eval(ctx, G, None, S)
            thc.thc_sync(ctx)
        finally:
            thc.thc_destroy(ctx)
        assert np.abs(S.cpu().numpy() - outs[0][i]).max() <= 1e-10 * max(1.0, np.abs(outs[0][i]).max())


def test_autotuner_table_and_cache(tmp_path):
    from paper_2404_17744_gb300 import thc
    cases = wb.make_batch(2, 30, 60, 4, 30.0, seed=9)
    _run_batch(cases, 1, tune=True, calls=1)
    n = thc.thc_autotune_entries()
    assert n > 0
    path = tmp_path / "tiles.txt"
    thc.thc_autotune_save(path)
    lines = open(path).read().split("\n")
    assert sum(1 for l in lines if l.strip()) == n
    choices = [(int(l.split()[0]), int(l.split()[-1])) for l in lines if l.strip()]
    bcd = [c for k, c in choices if k == thc.THC_KCLASS_SOX_BCD]
    assert bcd and all(c in (11, 12, 22) for c in bcd)            # cluster shapes of the B C/D blocks
    assert all(c in (128, 256) for k, c in choices if k != thc.THC_KCLASS_SOX_BCD)
    thc.thc_autotune_load(path)
    assert thc.thc_autotune_entries() == n
