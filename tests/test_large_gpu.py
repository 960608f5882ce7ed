"""The paper's largest sizes (Sec. III: up to ~1100 AOs; here N = 5 n).

* 500 AOs, 2500 THC points, tau = 0.1 and beta - 0.1: the 3 x BF16 path against the FP64
  GPU path (itself pinned to the oracle in test_sigma_gpu.py), 1e-6 bound,
  plus Sigma_ij = Sigma_ji;
* 1100 AOs, 5500 THC points, the same two tau points: the 3 x BF16 path alone (the FP64
  path needs about two minutes per tau point there): symmetry and a non-trivial
  result.
"""
import numpy as np
import pytest

from workloads import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _edge_case(name):
    """The workload with two tau points next to 0 and beta, where Sigma is largest."""
    case = synth.make_workload(name, n_tau=2)
    case.tau = np.array([0.1, case.beta - 0.1])
    case.tau_w = np.array([0.1, 0.1])
    case.G_tau = synth.noninteracting_G(case.F, case.S, 0.0, case.beta, case.tau)
    case.G_bmt = case.G_tau[::-1].copy()
    return case


def _eval(case, precision):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    ctx = thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, case.tau, precision, 3)
    try:
        G = torch.from_numpy(case.G_tau).to(dev)
        S = torch.empty_like(G)
        thc.thc_sigma_eval(ctx, G, None, S)
        E = thc.thc_energy(ctx, G, None, S, case.tau_w)
        thc.thc_sync(ctx)
        return S.cpu().numpy(), E
    finally:
        thc.thc_destroy(ctx)
        del X, V
        torch.cuda.empty_cache()


def test_500_ao_split_against_fp64():
    case = _edge_case("thc500")
    S64, E64 = _eval(case, 0)
    Ssp, Esp = _eval(case, 1)
    assert np.abs(S64 - np.swapaxes(S64, 1, 2)).max() <= 1e-10
    err = np.abs(Ssp - S64).max()
    print(f"500 AOs: max|Sigma| {np.abs(S64).max():.3e}, max|dSigma| split vs FP64 {err:.2e}, dE {abs(Esp - E64):.2e}")
    assert err <= 1e-6
    assert abs(Esp - E64) <= 1e-5


def test_1100_ao_split_runs_at_full_size():
    case = _edge_case("thc1100")
    S, E = _eval(case, 1)
    assert np.isfinite(S).all() and np.isfinite(E)
    assert np.abs(S - np.swapaxes(S, 1, 2)).max() <= 1e-6 * max(1e-12, np.abs(S).max()) + 1e-12
    print(f"1100 AOs: max|Sigma| {np.abs(S).max():.3e}, E_dyn {E:.6e}")
    assert np.abs(S).max() > 0
