"""Screened direct term (THC_GW: scGW, and scGWSOX with THC_SOX) against the oracle's
sigma_gw_thc (pinned by its weak-coupling limit, the one-orbital closed form and
symmetry in tests/test_oracle_pins.py).  Bars: FP64 path 1e-10 Ha in Sigma; THC_BF16X3
(split projections and back-transform, FP64 screening) 1e-6 Ha.  THC ranks above 128
exercise the blocked symmetric-sweep inverse of the screening (blocks of 64 pivots on
the upper triangle: 192 whole blocks, 300 and 600 a ragged last one)."""
import functools

import numpy as np
import pytest

from oracle import thc_oracle as o
from workloads import ir, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def _grid(beta, wmax):
    g = ir.make_loop_grid(beta, wmax)
    return g, ir.make_bosonic_transforms(g)


def _run(case, g, bt, terms, G, precision=0):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    ctx = thc.thc_sigma_init(case.n, case.N, len(g.tau), g.basis.beta, X, V, g.tau, precision, terms,
                             torch.cuda.current_stream(dev).cuda_stream)
    try:
        thc.thc_sigma_set_bosonic(ctx, bt.to_iw, bt.to_tau)
        Gd = torch.from_numpy(G).to(dev)
        S = torch.empty_like(Gd)
        thc.thc_sigma_eval(ctx, Gd, None, S)
        thc.thc_sync(ctx)
        return S.cpu().numpy()
    finally:
        thc.thc_destroy(ctx)


@functools.lru_cache(maxsize=None)
def _refs(n, N, seed):
    g, bt = _grid(50.0, 10.0)
    case = synth.make_sigma_case(n, N, 4, 50.0, seed, identity_S=False, n_occ=max(1, n // 3))
    G = synth.noninteracting_G(case.F, case.S, 0.0, 50.0, g.tau)
    Gb = G[::-1].copy()
    ref_gw = o.sigma_gw_thc(case.X, case.V, G, Gb, bt.to_iw, bt.to_tau)
    ref_sox = o.sigma_thc(case.X, case.V, G, Gb, terms="sox")
    ref_2 = o.sigma_thc(case.X, case.V, G, Gb, terms="direct")
    return case, G, ref_gw, ref_sox, ref_2


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
@pytest.mark.parametrize("n,N,seed", [(8, 30, 3), (21, 67, 4), (40, 150, 5), (24, 192, 7), (36, 300, 6), (40, 600, 9)])
def test_gw_and_gwsox_match_oracle(n, N, seed, precision, tol):
    from paper_2404_17744_gb300 import thc
    g, bt = _grid(50.0, 10.0)
    case, G, ref_gw, ref_sox, ref_2 = _refs(n, N, seed)
    S_gw = _run(case, g, bt, thc.THC_GW, G, precision)
    S_gwsox = _run(case, g, bt, thc.THC_GW | thc.THC_SOX, G, precision)
    e1 = np.abs(S_gw - ref_gw).max()
    e2 = np.abs(S_gwsox - (ref_gw + ref_sox)).max()
    print(f"GW p{precision} n={n} N={N}: max|dSigma| {e1:.2e} (GW+SOX {e2:.2e}); max|Sigma^GW| "
          f"{np.abs(ref_gw).max():.2e}, screening changes the second-order term by {np.abs(ref_gw - ref_2).max():.2e}")
    assert e1 <= tol and e2 <= tol
    assert np.abs(ref_gw - ref_2).max() > 1e-6 * np.abs(ref_2).max()


def test_gw_rejected_where_not_built():
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    case = synth.make_sigma_case(6, 14, 4, 50.0, 1)
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    with pytest.raises(thc.ThcError) as ei:
        thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, case.tau, thc.THC_FP64,
                           thc.THC_GW | thc.THC_DIRECT)
    assert ei.value.code == thc.THC_EINVAL
    ctx = thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, case.tau, thc.THC_FP64, thc.THC_GW)
    try:
        G = torch.from_numpy(case.G_tau).to(dev)
        with pytest.raises(thc.ThcError) as ei:   # no bosonic transforms yet
            thc.thc_sigma_eval(ctx, G, None, torch.empty_like(G))
        assert ei.value.code == thc.THC_EINVAL
    finally:
        thc.thc_destroy(ctx)
