"""Checkpoint / resume of the self-consistent loop and its per-iteration JSON-lines
metrics (host control around the library's kernels).

* A run interrupted after a few iterations, saved, and resumed in a new loop object
  (and a new proposer) continues with the same iterates: FP64 energies of every
  iteration within 1e-12 of the uninterrupted run and the same iteration count;
  with damping plus an online-trained proposal, the same converged energy within
  1e-9 Ha.
* The metrics file has one JSON line per iteration with the energy, its change,
  mu, the electron count, the residual and the per-kernel-class GPU times.
* A checkpoint of another loop (other sizes) is refused.
* run_loop(LoopConfig) reproduces the hand-built loop, resumes from its checkpoint,
  keeps the autotuner cache and runs the scGWSOX method.
"""
import json

import numpy as np
import pytest

from workloads import ir, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case():
    return synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)


def _grid():
    return ir.make_loop_grid(100.0, 10.0)


def test_resume_continues_the_same_iterates(tmp_path):
    from paper_2404_17744_gb300 import scf, thc
    case, g = _case(), _grid()
    A = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64)
    thc.thc_profile(A.ctx, True)
    try:
        assert A.run(tol=1e-10, max_iter=60, metrics=str(tmp_path / "a.jsonl"))
        ref = [r.E for r in A.records]
    finally:
        A.close()
    ck = str(tmp_path / "loop.npz")
    B = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64)
    try:
        assert not B.run(tol=1e-10, max_iter=4, checkpoint=ck)
    finally:
        B.close()
    C = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64)
    try:
        C.resume(ck)
        assert C.iteration == 4 and len(C.records) == 4
        assert C.run(tol=1e-10, max_iter=60)
        got = [r.E for r in C.records]
    finally:
        C.close()
    print(f"uninterrupted {len(ref)} iterations, resumed after 4: {len(got)}; "
          f"max |dE| {np.abs(np.array(ref) - np.array(got)).max():.2e}")
    assert len(got) == len(ref)
    assert np.abs(np.array(ref) - np.array(got)).max() <= 1e-12

    lines = [json.loads(x) for x in open(tmp_path / "a.jsonl")]
    assert [d["iter"] for d in lines] == list(range(1, len(ref) + 1))
    assert lines[0]["dE"] is None and abs(lines[-1]["dE"]) < 1e-10
    for d in lines:
        assert {"E", "E_dyn", "mu", "n_per_spin", "residual", "proposal", "kernel_ms"} <= set(d)
        assert abs(d["n_per_spin"] - 8.0) < 1e-6
    assert lines[0]["kernel_ms"].get("sox_B", 0.0) > 0.0   # FP64 SOX B step timed in the iteration


def test_resume_with_learned_proposer(tmp_path):
    from paper_2404_17744_gb300 import scf, thc
    case, g = _case(), _grid()

    def loop():
        return scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64, mixing="damp")

    A = loop()
    P = scf.LearnedProposer(A, max_proposals=3)
    try:
        assert A.run(tol=1e-9, max_iter=120, proposer=P)
        E_ref, n_ref, prop_ref = A.records[-1].E, len(A.records), P.proposed
    finally:
        P.close()
        A.close()
    ck = str(tmp_path / "learned.npz")
    B = loop()
    P = scf.LearnedProposer(B, max_proposals=3)
    try:
        B.run(tol=1e-9, max_iter=5, proposer=P, checkpoint=ck)
        assert P.proposed >= 1   # the interrupted part already trained and proposed
        count_b = thc.thc_proposer_count(P.p)
    finally:
        P.close()
        B.close()
    C = loop()
    P = scf.LearnedProposer(C, max_proposals=3, seed=1)   # other initial weights: the state replaces them
    try:
        C.resume(ck, proposer=P)
        assert thc.thc_proposer_count(P.p) == count_b and P.proposed >= 1
        assert C.run(tol=1e-9, max_iter=120, proposer=P)
        E, n, prop = C.records[-1].E, len(C.records), P.proposed
    finally:
        P.close()
        C.close()
    print(f"uninterrupted: {n_ref} iterations, {prop_ref} proposals, E {E_ref:.12f}; "
          f"resumed: {n} iterations, {prop} proposals, E {E:.12f}")
    assert abs(E - E_ref) <= 1e-9
    assert abs(n - n_ref) <= 1 and prop == prop_ref


def test_checkpoint_of_another_loop_is_refused(tmp_path):
    from paper_2404_17744_gb300 import scf, thc
    case, g = _case(), _grid()
    small = synth.make_sigma_case(6, 14, 4, 100.0, 31, identity_S=False, n_occ=3)
    ck = str(tmp_path / "small.npz")
    S = scf.GF2Loop(small.X, small.V, small.F, small.S, g, 3.0, precision=thc.THC_FP64)
    try:
        S.run(tol=1e-10, max_iter=2, checkpoint=ck)
    finally:
        S.close()
    L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64)
    try:
        with pytest.raises(ValueError):
            L.resume(ck)
        assert L.iteration == 0
    finally:
        L.close()


def test_run_loop_from_config(tmp_path):
    """run_loop(config) gives the loop of the same knobs set by hand, resumes from its
    checkpoint, writes its metrics and saves the autotuner cache; the scGWSOX method runs
    with the bosonic transforms."""
    from paper_2404_17744_gb300 import scf, thc
    from paper_2404_17744_gb300.config import LoopConfig, run_loop
    case, g = _case(), _grid()
    cfg = LoopConfig(precision="fp64", mixing="diis", tol=1e-10, max_iter=60,
                     checkpoint=str(tmp_path / "c.npz"), metrics=str(tmp_path / "c.jsonl"))
    conv, recs = run_loop(case.X, case.V, case.F, case.S, g, 8.0, cfg)
    L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64)
    try:
        assert L.run(tol=1e-10, max_iter=60)
        ref = [r.E for r in L.records]
    finally:
        L.close()
    assert conv and [r.E for r in recs] == ref
    assert len(open(tmp_path / "c.jsonl").read().splitlines()) == len(ref)
    # a run cut short and resumed from the checkpoint by a second call
    short = LoopConfig(**{**cfg.__dict__, "max_iter": 3, "metrics": None})
    assert not run_loop(case.X, case.V, case.F, case.S, g, 8.0, short)[0]
    conv2, recs2 = run_loop(case.X, case.V, case.F, case.S, g, 8.0, LoopConfig(**{**cfg.__dict__, "metrics": None}),
                            resume=True)
    assert conv2 and [r.E for r in recs2] == ref
    # 3xBF16 with the autotuner cache; scGWSOX with the screened term
    tiles = tmp_path / "tiles.txt"
    c3 = LoopConfig(precision="bf16x3", mixing="damp", tol=1e-6, max_iter=80, learned_proposals=1,
                    autotune_cache=str(tiles))
    conv3, recs3 = run_loop(case.X, case.V, case.F, case.S, g, 8.0, c3)
    assert conv3 and tiles.exists() and abs(recs3[-1].E - ref[-1]) < 1e-5
    cg = LoopConfig(method="gwsox", tol=1e-10, max_iter=60)
    with pytest.raises(ValueError):
        run_loop(case.X, case.V, case.F, case.S, g, 8.0, cg)
    conv4, recs4 = run_loop(case.X, case.V, case.F, case.S, g, 8.0, cg, bosonic=ir.make_bosonic_transforms(g))
    assert conv4 and abs(recs4[-1].E - ref[-1]) > 1e-7   # the screening moves the energy
