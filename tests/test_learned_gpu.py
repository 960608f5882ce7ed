"""GPU checks of the learned-proposal network and of its use in the loop.

* forward pass and gradients of the project's MLP kernels against the FP64
  oracle evaluated with the same FP16 working weights;
* Adam training lowers the loss of a regression the network can represent;
* a loop with learned proposals converges to the same energy as the loop
  without them (the proposals never change the fixed point); the iteration
  counts with and without proposals are printed.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as mo
from workloads import ir, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _weights(rng, din, H, dout):
    return (rng.standard_normal((H, din)).astype(np.float32) * np.float32(np.sqrt(2.0 / din)),
            (rng.standard_normal(H) * 0.1).astype(np.float32),
            rng.standard_normal((dout, H)).astype(np.float32) * np.float32(np.sqrt(1.0 / H)),
            (rng.standard_normal(dout) * 0.1).astype(np.float32))


@pytest.mark.parametrize("B,din,H,dout", [(5, 3, 7, 2), (300, 104, 512, 52), (1000, 20, 65, 33)])
def test_mlp_forward_and_gradients_match_oracle(B, din, H, dout):
    from paper_2404_17744_gb300 import thc
    rng = np.random.default_rng(B)
    W1, b1, W2, b2 = _weights(rng, din, H, dout)
    X = rng.standard_normal((B, din)).astype(np.float32)
    T = rng.standard_normal((B, dout)).astype(np.float32)
    dev = torch.device("cuda:0")
    m = thc.thc_mlp_init(din, H, dout, B, W1, b1, W2, b2)
    try:
        Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
        Yd = torch.empty((B, dout), dtype=torch.float32, device=dev)
        thc.thc_mlp_forward(m, B, Xd, Yd)
        torch.cuda.synchronize()
        Y_ref, _ = mo.forward(X, W1, b1, W2, b2, fp16_weights=True)
        assert np.abs(Yd.cpu().numpy() - Y_ref).max() <= 1e-4 * max(1.0, np.abs(Y_ref).max())
        g = [np.empty_like(a) for a in (W1, b1, W2, b2)]
        loss = thc.thc_mlp_gradients(m, B, Xd, Td, *g)
        ref = mo.loss_and_grads(X, T, W1, b1, W2, b2, fp16_weights=True)
        assert abs(loss - ref[0]) <= 1e-5 * abs(ref[0])
        for got, want in zip(g, ref[1:]):
            assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max() + 1e-7
    finally:
        thc.thc_mlp_destroy(m)


def test_mlp_training_lowers_loss():
    from paper_2404_17744_gb300 import thc
    rng = np.random.default_rng(9)
    B, din, H, dout = 4096, 16, 128, 8
    A = rng.standard_normal((dout, din)) / np.sqrt(din)
    X = rng.standard_normal((B, din)).astype(np.float32)
    T = (X @ A.T + 0.3 * np.maximum(X[:, :dout], 0)).astype(np.float32)
    W1, b1, W2, b2 = _weights(rng, din, H, dout)
    dev = torch.device("cuda:0")
    m = thc.thc_mlp_init(din, H, dout, B, W1, b1, W2, b2)
    try:
        Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
        l0 = thc.thc_mlp_gradients(m, B, Xd, Td)
        l1 = thc.thc_mlp_train(m, B, Xd, Td, 400, 1024, 3e-3)
        l2 = thc.thc_mlp_gradients(m, B, Xd, Td)
        print(f"loss {l0:.3e} -> {l2:.3e} (last mini-batch {l1:.3e})")
        assert l2 < 0.05 * l0
    finally:
        thc.thc_mlp_destroy(m)


@pytest.mark.parametrize("precision,tol,bar", [(0, 1e-10, 1e-9), (1, 1e-6, 1e-5)])
def test_loop_with_learned_proposals_reaches_the_same_energy(precision, tol, bar):
    from paper_2404_17744_gb300 import scf
    case = synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)
    g = ir.make_loop_grid(100.0, 10.0)
    runs = {}
    for learned in (False, True):
        L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=precision)
        P = scf.LearnedProposer(L) if learned else None
        try:
            conv = L.run(tol=tol, max_iter=80, proposer=P)
            runs[learned] = (conv, L.records, (P.accepted, P.rejected) if P else None)
        finally:
            if P:
                P.close()
            L.close()
    (c0, r0, _), (c1, r1, ar) = runs[False], runs[True]
    print(f"precision {precision}: plain {len(r0)} iterations E {r0[-1].E:.10f}; learned {len(r1)} iterations "
          f"E {r1[-1].E:.10f}, proposals accepted/rejected {ar}; labels {[r.proposal for r in r1]}")
    assert c0 and c1
    assert abs(r0[-1].E - r1[-1].E) < bar


@pytest.mark.parametrize("precision,tol,bar", [(0, 1e-10, 1e-9), (1, 1e-6, 1e-5)])
def test_transfer_between_related_systems(precision, tol, bar):
    """Fit on the trajectory of one system, propose for a related one (same sizes,
    another seed); the converged energy is unchanged and the iteration counts with
    and without the transferred network are printed."""
    from paper_2404_17744_gb300 import scf
    g = ir.make_loop_grid(100.0, 10.0)
    a = synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)
    b = synth.make_sigma_case(20, 60, 4, 100.0, 17746, identity_S=False, n_occ=8)
    LA = scf.GF2Loop(a.X, a.V, a.F, a.S, g, 8.0, precision=precision)
    P = scf.LearnedProposer(LA, record=True, steps=400)
    try:
        assert LA.run(tol=tol, max_iter=80, proposer=P)
        loss = P.fit()
        P.start_transfer()
        runs = {}
        for learned in (False, True):
            LB = scf.GF2Loop(b.X, b.V, b.F, b.S, g, 8.0, precision=precision)
            try:
                conv = LB.run(tol=tol, max_iter=80, proposer=P if learned else None)
                runs[learned] = (conv, LB.records)
            finally:
                LB.close()
    finally:
        P.close()
        LA.close()
    (c0, r0), (c1, r1) = runs[False], runs[True]
    print(f"transfer precision {precision}: fit loss {loss:.3e}; plain {len(r0)} iterations, learned {len(r1)} "
          f"(accepted {P.accepted}, rejected {P.rejected}); labels {[r.proposal for r in r1]}")
    assert c0 and c1
    assert abs(r0[-1].E - r1[-1].E) < bar


def test_learned_proposals_cut_damped_iterations():
    """What the trained network gains over the method without it: the loop's damped
    fixed-point iteration (damping 0.5 throughout) reaches |dE| < 1e-9 in fewer Sigma
    evaluations when the online-trained network proposes every few iterations (it
    extrapolates the per-element IR-coefficient trajectories towards their limit), and
    to the same energy.  DIIS needs fewer iterations still; the counts are printed."""
    from paper_2404_17744_gb300 import scf
    case = synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)
    g = ir.make_loop_grid(100.0, 10.0)
    out = {}
    for name, mixing, kw in (("damped", "damp", None),
                             ("damped+learned", "damp", dict(max_proposals=8, cooldown=1, active_above=1e-9)),
                             ("diis", "diis", None)):
        L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=0, mixing=mixing)
        P = scf.LearnedProposer(L, **kw) if kw is not None else None
        try:
            conv = L.run(tol=1e-9, max_iter=120, proposer=P)
            out[name] = (conv, len(L.records), L.records[-1].E)
        finally:
            if P:
                P.close()
            L.close()
    print("Sigma evaluations to |dE| < 1e-9: " + ", ".join(f"{k} {v[1]}" for k, v in out.items()))
    assert all(v[0] for v in out.values())
    assert out["damped+learned"][1] <= 0.8 * out["damped"][1]
    assert abs(out["damped+learned"][2] - out["damped"][2]) < 1e-8
