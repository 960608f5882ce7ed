"""GPU parity of the FP64 path against the FP64 CPU oracle, through the C ABI.

Bar: max-abs difference <= 1e-10 Ha in Sigma and in E_dyn (FP64 path).
"""
import os

import numpy as np
import pytest

from oracle import thc_oracle as o
from workloads import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-10


def _run(case, precision=0, terms=3, explicit_bmt=False, host=False):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    X = torch.from_numpy(case.X).to(dev)
    V = torch.from_numpy(case.V).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    ctx = thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, np.ascontiguousarray(case.tau),
                             precision, terms, stream)
    try:
        if host:
            S = np.empty_like(case.G_tau)
            thc.thc_sigma_eval_host(ctx, np.ascontiguousarray(case.G_tau),
                                    np.ascontiguousarray(case.G_bmt) if explicit_bmt else None, S)
            return S, None
        G = torch.from_numpy(case.G_tau).to(dev)
        Gb = torch.from_numpy(np.ascontiguousarray(case.G_bmt)).to(dev) if explicit_bmt else None
        S = torch.empty_like(G)
        thc.thc_sigma_eval(ctx, G, Gb, S)
        E = thc.thc_energy(ctx, G, Gb, S, np.ascontiguousarray(case.tau_w))
        torch.cuda.synchronize()
        return S.cpu().numpy(), E
    finally:
        thc.thc_destroy(ctx)


def _oracle(case, terms="both"):
    S = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt, terms=terms)
    return S, o.energy_dyn_tau(case.G_bmt, S, case.tau_w)


def test_thc20_workload_parity():
    case = synth.make_workload("thc20")
    S, E = _run(case)
    R, ER = _oracle(case)
    assert np.abs(S - R).max() <= TOL
    assert abs(E - ER) <= TOL


@pytest.mark.parametrize("n,N,n_tau,seed", [(37, 131, 6, 1), (65, 67, 4, 2), (1, 1, 2, 3), (3, 200, 3, 4),
                                             (64, 128, 2, 5), (130, 70, 2, 6)])
def test_ragged_sizes_parity(n, N, n_tau, seed):
    case = synth.make_sigma_case(n, N, n_tau, 30.0, seed)
    S, E = _run(case)
    R, ER = _oracle(case)
    assert np.abs(S - R).max() <= TOL
    assert abs(E - ER) <= TOL


@pytest.mark.parametrize("terms,name", [(1, "direct"), (2, "sox")])
def test_single_terms_parity(terms, name):
    case = synth.make_sigma_case(21, 75, 4, 40.0, 9, n_occ=8)
    S, E = _run(case, terms=terms)
    R, ER = _oracle(case, terms=name)
    assert np.abs(S - R).max() <= TOL
    assert abs(E - ER) <= TOL


def test_non_mirrored_grid_needs_and_uses_G_bmt():
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(11, 30, 5, 25.0, 13, identity_S=False, n_occ=5)
    rng = np.random.default_rng(3)
    tau = np.sort(rng.uniform(0.5, 24.5, size=5))
    case.tau = tau
    case.tau_w = np.full(5, 0.1)
    case.G_tau = synth.noninteracting_G(case.F, case.S, 0.0, case.beta, tau)
    case.G_bmt = synth.noninteracting_G(case.F, case.S, 0.0, case.beta, case.beta - tau)
    with pytest.raises(thc.ThcError) as ei:
        _run(case)
    assert ei.value.code == thc.THC_EINVAL
    S, E = _run(case, explicit_bmt=True)
    R, ER = _oracle(case)
    assert np.abs(S - R).max() <= TOL
    assert abs(E - ER) <= TOL


def test_small_workspace_blocking_matches(monkeypatch):
    case = synth.make_sigma_case(40, 150, 5, 30.0, 17)
    monkeypatch.setenv("THC_WORKSPACE_BYTES", str(600_000))   # forces several P blocks and tau chunks of 1
    S, E = _run(case)
    R, ER = _oracle(case)
    assert np.abs(S - R).max() <= TOL
    assert abs(E - ER) <= TOL


def test_host_entry_point_matches_device():
    case = synth.make_sigma_case(33, 90, 4, 30.0, 19)
    Sd, _ = _run(case)
    Sh, _ = _run(case, host=True)
    assert np.array_equal(Sd, Sh)


def test_deterministic_repeat():
    case = synth.make_sigma_case(50, 160, 3, 30.0, 23)
    S1, E1 = _run(case)
    S2, E2 = _run(case)
    assert np.array_equal(S1, S2) and E1 == E2


def test_thc200_full_size_sampled_parity():
    """200 AOs, 1000 THC points, 100 tau points (the bench workload, same launch
    configuration): Sigma at sampled tau points against the oracle, symmetry at all."""
    case = synth.make_workload("thc200")
    S, E = _run(case)
    assert np.abs(S - np.swapaxes(S, 1, 2)).max() <= TOL
    U = o.thc_U(case.X, case.V)
    for k in (0, 37, 99):
        G = case.G_tau[k]
        Gm = o.g_minus_tau(case.G_bmt[k])
        R = o.sigma_sox_thc(case.X, U, G, Gm) + o.sigma_direct_thc(case.X, case.V, G, Gm)
        assert np.abs(S[k] - R).max() <= TOL, k
    # energy reduction of the GPU Sigma against a host trace of the same Sigma
    E_host = o.energy_dyn_tau(case.G_bmt, S, case.tau_w)
    assert abs(E - E_host) <= 1e-12 * max(1.0, abs(E_host))
