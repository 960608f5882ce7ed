"""thc_energy_static: the energy entry point for callers that cannot allocate
device memory (an external allocator owns the GPU, or allocation is not
allowed after start-up).  Its scratch is a fixed static device array, so the
test checks that two calls in a row, on different inputs, each reproduce the
context-based thc_energy, and that sizes beyond the array are rejected.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from workloads import synth


def test_static_energy_rejects_oversized_grid():
    from paper_2404_17744_gb300 import build, thc
    import os
    if not os.path.exists(thc.LIB_PATH):
        build.build()
    n_tau = 4097   # THC_STATIC_MAX_TAU + 1
    w = np.zeros(n_tau)
    with pytest.raises(thc.ThcError) as ei:
        thc.thc_energy_static(3, n_tau, 1, None, 2, w)
    assert ei.value.code == thc.THC_EINVAL
    assert "static scratch limit" in thc.thc_last_error(None)


@pytest.mark.gpu
def test_static_energy_matches_context_energy_twice():
    torch = pytest.importorskip("torch")
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [synth.make_sigma_case(23, 70, 12, 30.0, 41, n_occ=9),
             synth.make_sigma_case(17, 40, 6, 20.0, 42, identity_S=False, n_occ=6)]
    for case in cases:   # two calls in a row; the second has fewer tau points than the first
        X = torch.from_numpy(case.X).to(dev)
        V = torch.from_numpy(case.V).to(dev)
        G = torch.from_numpy(case.G_tau).to(dev)
        S = torch.empty_like(G)
        ctx = thc.thc_sigma_init(case.n, case.N, case.n_tau, case.beta, X, V, case.tau,
                                 thc.THC_FP64, thc.THC_DIRECT | thc.THC_SOX, stream)
        try:
            thc.thc_sigma_eval(ctx, G, None, S)
            E_ctx = thc.thc_energy(ctx, G, None, S, case.tau_w)
        finally:
            thc.thc_destroy(ctx)
        E_static = thc.thc_energy_static(case.n, case.n_tau, G, None, S, case.tau_w, stream)
        # same kernels' arithmetic in the same order as the context path: equal bit for bit
        assert E_static == E_ctx
        Gb = torch.flip(G, dims=[0]).contiguous()   # explicit G(beta - tau) gives the same number
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        E_static_b = thc.thc_energy_static(case.n, case.n_tau, G, Gb, S, case.tau_w, stream)
        assert torch.cuda.mem_get_info(dev)[0] == free_before   # the call allocated nothing
        assert E_static_b == E_ctx
