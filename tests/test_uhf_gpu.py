"""Spin-unrestricted evaluation (thc_sigma_eval_uhf) against the FP64 oracle.

The oracle's unrestricted THC route is pinned to the spin-orbital four-index
definition (tests/test_oracle_pins.py).  Bars as for the restricted path: FP64
1e-10 Ha in Sigma and E_dyn, THC_BF16X3 1e-6 Ha in Sigma and 1e-5 Ha in E_dyn.
With G_a = G_b the unrestricted result must equal the restricted one bit for bit
(the summed polarisation is exactly twice the single-spin one).
"""
import numpy as np
import pytest

from oracle import thc_oracle as o
from workloads import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _spin_pair(n, N, n_tau, beta, seed, terms=3):
    """A case whose beta spin has one electron fewer than its alpha spin (mu moved
    between the two highest occupied levels)."""
    case = synth.make_sigma_case(n, N, n_tau, beta, seed, identity_S=False, n_occ=max(1, n // 3))
    k = max(1, n // 3)
    mu_b = 0.5 * (case.eps[k - 2] + case.eps[k - 1]) if k >= 2 else case.eps[0] - 0.5
    Gb = synth.noninteracting_G(case.F, case.S, mu_b, beta, case.tau)
    return case, case.G_tau, Gb


def _oracle(case, Ga, Gb, terms):
    U = o.thc_U(case.X, case.V)
    nt = case.n_tau
    Sa = np.empty_like(Ga)
    Sb = np.empty_like(Gb)
    for k in range(nt):
        args = (Ga[k], Gb[k], -Ga[nt - 1 - k], -Gb[nt - 1 - k])
        if terms == 3:
            Sa[k], Sb[k] = o.sigma_uhf_thc(case.X, case.V, U, *args)
        else:
            # single terms: SOX per spin alone, or the bubble alone (V and U of the full route)
            a, b = o.sigma_uhf_thc(case.X, case.V, U, *args)
            xa = o.sigma_sox_thc(case.X, U, Ga[k], -Ga[nt - 1 - k])
            xb = o.sigma_sox_thc(case.X, U, Gb[k], -Gb[nt - 1 - k])
            Sa[k], Sb[k] = (xa, xb) if terms == 2 else (a - xa, b - xb)
    return Sa, Sb


def _gpu(case, Ga, Gb, precision, terms=3):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    ctx = thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, case.tau, precision, terms,
                             torch.cuda.current_stream(dev).cuda_stream)
    try:
        ga = torch.from_numpy(np.ascontiguousarray(Ga)).to(dev)
        gb = torch.from_numpy(np.ascontiguousarray(Gb)).to(dev)
        sa, sb = torch.empty_like(ga), torch.empty_like(gb)
        thc.thc_sigma_eval_uhf(ctx, ga, None, gb, None, sa, sb)
        Ea = thc.thc_energy(ctx, ga, None, sa, case.tau_w)
        Eb = thc.thc_energy(ctx, gb, None, sb, case.tau_w)
        sr = torch.empty_like(ga)
        thc.thc_sigma_eval(ctx, ga, None, sr)
        thc.thc_sync(ctx)
        return sa.cpu().numpy(), sb.cpu().numpy(), 0.5 * (Ea + Eb), sr.cpu().numpy()
    finally:
        thc.thc_destroy(ctx)


@pytest.mark.parametrize("precision,s_tol,e_tol", [(0, 1e-10, 1e-10), (1, 1e-6, 1e-5)])
@pytest.mark.parametrize("n,N,n_tau,seed", [(20, 60, 8, 3), (37, 131, 6, 4), (70, 260, 4, 5)])
def test_uhf_matches_oracle(precision, s_tol, e_tol, n, N, n_tau, seed):
    case, Ga, Gb = _spin_pair(n, N, n_tau, 30.0, seed)
    Sa, Sb, E, _ = _gpu(case, Ga, Gb, precision)
    Ra, Rb = _oracle(case, Ga, Gb, 3)
    ER = o.energy_dyn_tau_uhf(Ga[::-1], Gb[::-1], Ra, Rb, case.tau_w)
    err = max(np.abs(Sa - Ra).max(), np.abs(Sb - Rb).max())
    print(f"uhf p{precision} n={n}: max|dSigma| {err:.2e} (max|Sigma| {np.abs(Ra).max():.2e}), |dE| {abs(E - ER):.2e}")
    assert np.abs(Ra - Rb).max() > 1e-3 * np.abs(Ra).max()   # the spins really differ
    assert err <= s_tol and abs(E - ER) <= e_tol


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("terms", [1, 2])
def test_uhf_single_terms(precision, terms):
    case, Ga, Gb = _spin_pair(24, 80, 4, 30.0, 9)
    Sa, Sb, _, _ = _gpu(case, Ga, Gb, precision, terms)
    Ra, Rb = _oracle(case, Ga, Gb, terms)
    tol = 1e-10 if precision == 0 else 1e-6
    assert max(np.abs(Sa - Ra).max(), np.abs(Sb - Rb).max()) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_uhf_equal_spins_equal_restricted_bitwise(precision):
    case = synth.make_sigma_case(33, 100, 6, 30.0, 7, identity_S=False, n_occ=11)
    Sa, Sb, E, Sr = _gpu(case, case.G_tau, case.G_tau, precision)
    assert np.array_equal(Sa, Sr) and np.array_equal(Sb, Sr)
