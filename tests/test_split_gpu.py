"""GPU checks of the split-precision (3 x BF16, tcgen05) path.

* thc_gemm_bf16x3 against FP64 products: |C - A B^T| <= 4e-5 (|A| |B|^T) elementwise,
  the bound of three hi/lo BF16 products (about 2^-16 relative per product) with
  FP32 accumulation.
* Sigma(tau) and E_dyn of THC_BF16X3 against the FP64 oracle: max-abs <= 1e-6 Ha
  in Sigma and <= 1e-5 Ha in E_dyn; the error at every tau point is printed.
"""
import numpy as np
import pytest

from oracle import thc_oracle as o
from workloads import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIGMA_TOL = 1e-6
ENERGY_TOL = 1e-5


def _gemm(batch, M, N, K, bcast_a=False, seed=0):
    from paper_2404_17744_gb300 import thc
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((1 if bcast_a else batch, M, K))
    B = rng.standard_normal((batch, N, K))
    dev = torch.device("cuda:0")
    At = torch.from_numpy(A).to(dev)
    Bt = torch.from_numpy(B).to(dev)
    C = torch.zeros((batch, M, N), dtype=torch.float64, device=dev)
    thc.thc_gemm_bf16x3(batch, M, N, K, At, 0 if bcast_a else M * K, Bt, N * K, C, M * N,
                        torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    ref = np.matmul(A, np.swapaxes(B, 1, 2))
    bound = 4e-5 * np.matmul(np.abs(A), np.swapaxes(np.abs(B), 1, 2)) + 1e-30
    return C.cpu().numpy(), ref, bound


@pytest.mark.parametrize("batch,M,N,K,bcast", [(1, 128, 128, 64, False), (1, 200, 77, 100, False),
                                                (3, 300, 260, 200, False), (2, 129, 256, 130, True),
                                                (1, 1, 1, 1, False), (1, 64, 300, 1000, False)])
def test_gemm_bf16x3(batch, M, N, K, bcast):
    C, ref, bound = _gemm(batch, M, N, K, bcast)
    err = np.abs(C - ref)
    assert np.all(err <= bound), float((err / bound).max())
    # and it is not accidentally FP64-exact: the split really runs on BF16
    assert err.max() > 0


def _run(case, terms=3):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    ctx = thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, np.ascontiguousarray(case.tau),
                             thc.THC_BF16X3, terms, stream)
    try:
        G = torch.from_numpy(case.G_tau).to(dev)
        S = torch.empty_like(G)
        thc.thc_sigma_eval(ctx, G, None, S)
        E = thc.thc_energy(ctx, G, None, S, np.ascontiguousarray(case.tau_w))
        thc.thc_sync(ctx)
        return S.cpu().numpy(), E
    finally:
        thc.thc_destroy(ctx)


def _check(case, terms=3, name="both"):
    S, E = _run(case, terms)
    R = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt, terms=name)
    ER = o.energy_dyn_tau(case.G_bmt, R, case.tau_w)
    per_tau = np.abs(S - R).max(axis=(1, 2))
    print("max|dSigma| per tau:", " ".join(f"{x:.1e}" for x in per_tau), f"|dE| = {abs(E - ER):.2e}")
    assert per_tau.max() <= SIGMA_TOL
    assert abs(E - ER) <= ENERGY_TOL
    return per_tau, abs(E - ER)


def test_split_thc20_workload():
    _check(synth.make_workload("thc20"))


# n around the 64-column K blocks (a shallow last block is loaded in 16- or 32-column
# boxes), the 128-row q blocks of the A contraction and its 256-column v blocks
@pytest.mark.parametrize("n,N,n_tau,seed", [(37, 131, 6, 1), (65, 67, 4, 2), (1, 1, 2, 3), (130, 70, 2, 6),
                                            (63, 70, 2, 7), (64, 96, 2, 8), (96, 100, 2, 12), (129, 140, 2, 9),
                                            (257, 270, 2, 10)])
def test_split_ragged(n, N, n_tau, seed):
    _check(synth.make_sigma_case(n, N, n_tau, 30.0, seed))


@pytest.mark.parametrize("terms,name", [(1, "direct"), (2, "sox")])
def test_split_single_terms(terms, name):
    _check(synth.make_sigma_case(21, 75, 4, 40.0, 9, n_occ=8), terms, name)


@pytest.mark.parametrize("budget", [2_000_000, 300_000])
def test_split_small_workspace(monkeypatch, budget):
    # 300 kB gives P blocks of 23 THC points: the fused B C/D kernel then starts its blocks
    # at P0 that are not multiples of its 128-row tiles, and D's upper triangle crosses them
    monkeypatch.setenv("THC_WORKSPACE_BYTES", str(budget))
    _check(synth.make_sigma_case(40, 150, 5, 30.0, 17))


def test_split_thc200_sampled():
    case = synth.make_workload("thc200")
    S, E = _run(case)
    U = o.thc_U(case.X, case.V)
    for k in (0, 37, 99):
        G = case.G_tau[k]
        Gm = o.g_minus_tau(case.G_bmt[k])
        R = o.sigma_sox_thc(case.X, U, G, Gm) + o.sigma_direct_thc(case.X, case.V, G, Gm)
        err = np.abs(S[k] - R).max()
        print(f"tau[{k}] max|dSigma| = {err:.2e}  max|Sigma| = {np.abs(R).max():.2e}")
        assert err <= SIGMA_TOL
