"""Screened direct term (THC_GW: scGW, and scGWSOX with THC_SOX) against the oracle's
sigma_gw_thc (pinned by its weak-coupling limit, the one-orbital closed form and
symmetry in tests/test_oracle_pins.py), restricted and unrestricted (sigma_gw_uhf_thc,
pinned by its restricted limit, the unrestricted bubble at weak coupling and a
two-level one-orbital closed form).  Bars: FP64 path 1e-10 Ha in Sigma; THC_BF16X3
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


@functools.lru_cache(maxsize=None)
def _uhf_refs(n, N, seed):
    """Spin b with one electron fewer than spin a (mu between its two highest occupied
    levels), the oracle's unrestricted screened term and each spin's SOX."""
    g, bt = _grid(50.0, 10.0)
    k = max(2, n // 3)
    case = synth.make_sigma_case(n, N, 4, 50.0, seed, identity_S=False, n_occ=k)
    Ga = synth.noninteracting_G(case.F, case.S, 0.0, 50.0, g.tau)
    mu_b = 0.5 * (case.eps[k - 2] + case.eps[k - 1])
    Gb = synth.noninteracting_G(case.F, case.S, mu_b, 50.0, g.tau)
    ra, rb = o.sigma_gw_uhf_thc(case.X, case.V, Ga, Ga[::-1].copy(), Gb, Gb[::-1].copy(), bt.to_iw, bt.to_tau)
    sa = o.sigma_thc(case.X, case.V, Ga, Ga[::-1].copy(), terms="sox")
    sb = o.sigma_thc(case.X, case.V, Gb, Gb[::-1].copy(), terms="sox")
    return case, Ga, Gb, (ra, rb), (sa, sb)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
@pytest.mark.parametrize("n,N,seed", [(8, 30, 3), (21, 67, 4), (36, 300, 6)])
def test_uhf_gw_and_gwsox_match_oracle(n, N, seed, precision, tol):
    """thc_sigma_eval_uhf with THC_GW and THC_GW | THC_SOX against the oracle's
    unrestricted screened term (bubble over both spins, one W, outer line per spin),
    plus each spin's SOX; G(beta - tau) from the mirrored grid."""
    from paper_2404_17744_gb300 import thc
    g, bt = _grid(50.0, 10.0)
    case, Ga, Gb, gw, sox = _uhf_refs(n, N, seed)
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    Gad = torch.from_numpy(Ga).to(dev)
    Gbd = torch.from_numpy(Gb).to(dev)
    errs = []
    for terms, with_sox in ((thc.THC_GW, False), (thc.THC_GW | thc.THC_SOX, True)):
        ctx = thc.thc_sigma_init(case.n, case.N, len(g.tau), g.basis.beta, X, V, g.tau, precision, terms,
                                 torch.cuda.current_stream(dev).cuda_stream)
        try:
            thc.thc_sigma_set_bosonic(ctx, bt.to_iw, bt.to_tau)
            Sa = torch.empty_like(Gad)
            Sb = torch.empty_like(Gbd)
            thc.thc_sigma_eval_uhf(ctx, Gad, None, Gbd, None, Sa, Sb)
            thc.thc_sync(ctx)
            for s, S in enumerate((Sa, Sb)):
                ref = gw[s] + (sox[s] if with_sox else 0.0)
                errs.append(np.abs(S.cpu().numpy() - ref).max())
        finally:
            thc.thc_destroy(ctx)
    print(f"UHF GW p{precision} n={n} N={N}: max|dSigma| GW a/b {errs[0]:.2e}/{errs[1]:.2e}, "
          f"GW+SOX a/b {errs[2]:.2e}/{errs[3]:.2e}; spins differ by {np.abs(gw[0] - gw[1]).max():.2e}")
    assert max(errs) <= tol
    assert np.abs(gw[0] - gw[1]).max() > 1e-4 * np.abs(gw[0]).max()


def test_uhf_gw_equal_spins_is_the_restricted_result():
    """With G_a = G_b the unrestricted screened term equals the restricted one (the bubble
    accumulated over the two spins is twice the single-spin one, up to one rounding)."""
    from paper_2404_17744_gb300 import thc
    g, bt = _grid(50.0, 10.0)
    case, G, _, _, _ = _refs(21, 67, 4)
    R = _run(case, g, bt, thc.THC_GW | thc.THC_SOX, G)
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    Gd = torch.from_numpy(G).to(dev)
    ctx = thc.thc_sigma_init(case.n, case.N, len(g.tau), g.basis.beta, X, V, g.tau, 0, thc.THC_GW | thc.THC_SOX,
                             torch.cuda.current_stream(dev).cuda_stream)
    try:
        thc.thc_sigma_set_bosonic(ctx, bt.to_iw, bt.to_tau)
        Sa = torch.empty_like(Gd)
        Sb = torch.empty_like(Gd)
        thc.thc_sigma_eval_uhf(ctx, Gd, None, Gd, None, Sa, Sb)
        thc.thc_sync(ctx)
        a, b = Sa.cpu().numpy(), Sb.cpu().numpy()
    finally:
        thc.thc_destroy(ctx)
    assert np.array_equal(a, b)
    assert np.abs(a - R).max() <= 1e-14 * np.abs(R).max()


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
