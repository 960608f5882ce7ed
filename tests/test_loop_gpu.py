"""GPU parity of the self-consistency loop (Dyson step, energies, full loop)
against the FP64 oracle loop, through the C ABI (include/thc_dyson.h).

Bars: G(tau) and mu of one Dyson step within 1e-9; energies of the same
(G, Sigma) within 1e-12; converged loop energy within 1e-9 (FP64) and within
1e-5 Ha (3 x BF16 self-energy, loop stopped at |dE| < 1e-7) of the oracle loop.
"""
import functools

import numpy as np
import pytest

from oracle import scf_oracle as so
from oracle import thc_oracle as o
from workloads import ir, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def grid_for(beta, wmax):
    return ir.make_loop_grid(beta, wmax)


def _dyson(case, g):
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    S = torch.from_numpy(case.S).to(dev)
    F = torch.from_numpy(case.F).to(dev)
    d = thc.thc_dyson_init(case.n, len(g.tau), len(g.iw), g.basis.L, g.basis.beta, S, F, g.U_tau, g.fit_tau, g.U_iw,
                           g.fit_iw, g.iw, g.u_beta, g.u_zero, torch.cuda.current_stream(dev).cuda_stream)
    return d


def test_dyson_step_matches_oracle():
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(9, 25, 4, 50.0, 41, identity_S=False, n_occ=4)
    g = grid_for(50.0, 10.0)
    G0, mu0 = so.solve_dyson(g, case.S, case.F, None, 4.0, 0.0)
    U = o.thc_U(case.X, case.V)
    nt = len(g.tau)
    Sig = np.stack([o.sigma_sox_thc(case.X, U, G0[k], -G0[nt - 1 - k]) +
                    o.sigma_direct_thc(case.X, case.V, G0[k], -G0[nt - 1 - k]) for k in range(nt)])
    G_ref, mu_ref = so.solve_dyson(g, case.S, case.F, Sig, 4.0, mu0)
    d = _dyson(case, g)
    try:
        dev = torch.device("cuda:0")
        Gd = torch.empty((nt, case.n, case.n), dtype=torch.float64, device=dev)
        Sd = torch.from_numpy(Sig).to(dev)
        # the inversions and transforms at exactly the oracle's mu (a tolerance that accepts the
        # starting point returns after one evaluation) ...
        assert thc.thc_dyson_solve(d, None, 4.0, mu0, 10.0, Gd) == mu0
        assert np.abs(Gd.cpu().numpy() - G0).max() < 1e-10
        assert thc.thc_dyson_solve(d, Sd, 4.0, mu_ref, 10.0, Gd) == mu_ref
        assert np.abs(Gd.cpu().numpy() - G_ref).max() < 1e-10
        # ... and the search: the count is fixed; inside the gap mu (and G at large tau) move
        # only as far as the count's tolerance allows
        mu = thc.thc_dyson_solve(d, Sd, 4.0, 0.0, 1e-12, Gd)
        E_check, _, n_check = thc.thc_dyson_energy(d, Gd, Sd)
        assert abs(n_check - 4.0) < 1e-9
        assert abs(mu - mu_ref) < 1e-4
        E, trgf, n = thc.thc_dyson_energy(d, Gd, Sd)
        assert abs(E - so.energy_ir(g, Gd.cpu().numpy(), Sig)) < 1e-12
        assert abs(n - 4.0) < 1e-9
    finally:
        thc.thc_dyson_destroy(d)


@pytest.mark.parametrize("mirrored", [True, False])
def test_dyson_inversions_with_and_without_mirrored_frequencies(mirrored):
    """A 37-orbital Dyson step at the oracle's mu, on the IR grid (frequencies in pairs
    w, -w: the GPU inverts half of them and conjugates) and on the same grid without
    its first Matsubara point (no pairs: every frequency inverted)."""
    import dataclasses
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(37, 80, 4, 50.0, 43, identity_S=False, n_occ=11)
    g = grid_for(50.0, 10.0)
    if not mirrored:
        U_iw = g.U_iw[1:]
        g = dataclasses.replace(g, n=g.n[1:], iw=g.iw[1:], U_iw=U_iw, fit_iw=np.linalg.pinv(U_iw))
    G0, mu0 = so.solve_dyson(g, case.S, case.F, None, 11.0, 0.0)
    rng = np.random.default_rng(5)
    nt = len(g.tau)
    Sig = 0.05 * synth.random_symmetric(nt, case.n, rng) * np.exp(-np.linspace(0, 3, nt))[:, None, None]
    G_ref, mu_ref = so.solve_dyson(g, case.S, case.F, Sig, 11.0, mu0)
    d = _dyson(case, g)
    try:
        dev = torch.device("cuda:0")
        Gd = torch.empty((nt, case.n, case.n), dtype=torch.float64, device=dev)
        Sd = torch.from_numpy(Sig).to(dev)
        assert thc.thc_dyson_solve(d, Sd, 11.0, mu_ref, 10.0, Gd) == mu_ref
        err = np.abs(Gd.cpu().numpy() - G_ref).max()
        print(f"mirrored={mirrored}: {len(g.iw)} frequencies, max|dG| = {err:.1e}")
        assert err < 1e-10
    finally:
        thc.thc_dyson_destroy(d)


def test_dyson_step_at_200_orbitals_matches_oracle():
    """A 200-orbital Dyson step on the Lambda = 1e5 grid (96 Matsubara points in pairs: 48
    inverted, more than one wave of resident clusters, so the set runs as whole waves of
    one cluster size and the rest with another) with the oracle's second-order Sigma of
    the noninteracting G, at the oracle's mu; and the search from mu = 0 to its count."""
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(200, 40, 4, 100.0, 47, identity_S=False, n_occ=40)
    g = grid_for(100.0, 1000.0)
    nt = len(g.tau)
    G0, mu0 = so.solve_dyson(g, case.S, case.F, None, 40.0, 0.0)
    U = o.thc_U(case.X, case.V)
    Sig = np.stack([o.sigma_sox_thc(case.X, U, G0[k], -G0[nt - 1 - k]) +
                    o.sigma_direct_thc(case.X, case.V, G0[k], -G0[nt - 1 - k]) for k in range(nt)])
    G_ref, mu_ref = so.solve_dyson(g, case.S, case.F, Sig, 40.0, mu0)
    d = _dyson(case, g)
    try:
        dev = torch.device("cuda:0")
        Gd = torch.empty((nt, case.n, case.n), dtype=torch.float64, device=dev)
        Sd = torch.from_numpy(Sig).to(dev)
        assert thc.thc_dyson_solve(d, Sd, 40.0, mu_ref, 10.0, Gd) == mu_ref
        err = np.abs(Gd.cpu().numpy() - G_ref).max()
        mu = thc.thc_dyson_solve(d, Sd, 40.0, 0.0, 1e-11, Gd)
        _, _, n = thc.thc_dyson_energy(d, Gd, Sd)
        print(f"200 orbitals, {len(g.iw)} frequencies: max|dG| = {err:.1e}; searched mu {mu:.10f} "
              f"(oracle {mu_ref:.10f}), count {n:.12f}")
        assert err < 1e-10
        assert abs(n - 40.0) < 1e-9 and abs(mu - mu_ref) < 1e-4
    finally:
        thc.thc_dyson_destroy(d)


def test_vector_utilities():
    from paper_2404_17744_gb300 import thc
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(5)
    a, b, c = (rng.standard_normal(100003) for _ in range(3))
    ta, tb, tc = (torch.from_numpy(x).to(dev) for x in (a, b, c))
    scratch = torch.empty(512, dtype=torch.float64, device=dev)
    assert abs(thc.thc_vec_dot(len(a), ta, tb, scratch) - a @ b) < 1e-10
    out = torch.empty_like(ta)
    thc.thc_vec_lincomb([0.5, -2.0, 3.0], [ta, tb, tc], len(a), out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - (0.5 * a - 2 * b + 3 * c)).max() < 1e-13
    thc.thc_vec_lincomb([2.0, 1.0], [ta, tb], len(a), ta)   # output aliases an input
    torch.cuda.synchronize()
    assert np.abs(ta.cpu().numpy() - (2 * a + b)).max() < 1e-13


def _loop(case, g, n_elec, precision, tol=1e-10):
    from paper_2404_17744_gb300 import scf
    L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, n_elec, precision=precision)
    try:
        conv = L.run(tol=tol, max_iter=80)
        return conv, L.records
    finally:
        L.close()


@pytest.mark.parametrize("n,N,beta,n_occ,seed", [(6, 14, 50.0, 3, 31), (20, 60, 100.0, 8, 17745)])
def test_fp64_loop_matches_oracle_loop(n, N, beta, n_occ, seed):
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(n, N, 4, beta, seed, identity_S=False, n_occ=n_occ)
    g = grid_for(beta, 10.0)
    ref = so.run_loop(case, g, float(n_occ), tol=1e-10)
    conv, recs = _loop(case, g, float(n_occ), thc.THC_FP64)
    assert conv and ref["converged"]
    print(f"oracle E {ref['E']:.12f} ({ref['iters']} it)  GPU E {recs[-1].E:.12f} ({len(recs)} it)")
    assert abs(recs[-1].E - ref["E"]) < 1e-9
    assert abs(len(recs) - ref["iters"]) <= 2
    assert abs(recs[-1].mu - ref["mu"]) < 1e-4          # mu is loose inside the gap
    assert abs(recs[-1].n_per_spin - n_occ) < 1e-9
    for r, h in zip(recs[:5], ref["history"][:5]):
        assert abs(r.E - h["E"]) < 1e-9


def test_split_loop_reaches_fp64_energy():
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)
    g = grid_for(100.0, 10.0)
    c1, r64 = _loop(case, g, 8.0, thc.THC_FP64, tol=1e-9)
    # the BF16 rounding of G makes the split Sigma map step-like at ~2^-17 relative, so its
    # last iterates can cycle near 1e-8 Ha: the split loop stops at |dE| < 1e-7
    c2, rsp = _loop(case, g, 8.0, thc.THC_BF16X3, tol=1e-7)
    dE = [f"{abs(b.E - a.E):.1e}" for a, b in zip(rsp[:-1], rsp[1:])]
    print(f"FP64 E {r64[-1].E:.10f} ({len(r64)} it), split E {rsp[-1].E:.10f} ({len(rsp)} it), |dE| {dE[-6:]}")
    assert c1 and c2
    assert abs(r64[-1].E - rsp[-1].E) < 1e-5


def test_count_slope_and_commutator_match_oracle():
    """thc_dyson_count (N and the analytic dN/dmu of the Newton search) and
    thc_dyson_commutator (the CDIIS error vector) against the oracle's formulas."""
    from paper_2404_17744_gb300 import thc
    case = synth.make_sigma_case(9, 25, 4, 50.0, 41, identity_S=False, n_occ=4)
    g = grid_for(50.0, 10.0)
    G0, mu0 = so.solve_dyson(g, case.S, case.F, None, 4.0, 0.0)
    U = o.thc_U(case.X, case.V)
    nt = len(g.tau)
    Sig = np.stack([o.sigma_sox_thc(case.X, U, G0[k], -G0[nt - 1 - k]) +
                    o.sigma_direct_thc(case.X, case.V, G0[k], -G0[nt - 1 - k]) for k in range(nt)])
    Siw = so.sigma_iw(g, Sig)
    d = _dyson(case, g)
    try:
        dev = torch.device("cuda:0")
        Sd = torch.from_numpy(Sig).to(dev)
        for mu in (mu0, mu0 + 0.2, mu0 - 0.7):
            n_gpu, dn_gpu = thc.thc_dyson_count(d, Sd, mu)
            Giw = so.dyson_iw(g, case.S, case.F, Siw, mu)
            n_ref = so.electron_count(g, case.S, Giw)
            dn_ref = so.electron_count_slope(g, case.S, Giw)
            assert abs(n_gpu - n_ref) < 1e-11 and abs(dn_gpu - dn_ref) < 1e-9 * max(1.0, abs(dn_ref))
        # commutator: G of the last solve (here the Sigma = 0 solve at the oracle's mu0)
        Gd = torch.empty((nt, case.n, case.n), dtype=torch.float64, device=dev)
        assert thc.thc_dyson_solve(d, None, 4.0, mu0, 10.0, Gd) == mu0
        E = torch.empty((len(g.iw), case.n, case.n, 2), dtype=torch.float64, device=dev)
        thc.thc_dyson_commutator(d, Sd, E)
        G0iw = so.dyson_iw(g, case.S, case.F, np.zeros_like(Siw), mu0)
        e_ref = so.commutator_residual(g, case.S, case.F, G0iw, Sig)
        e_gpu = E.cpu().numpy()
        e_gpu = e_gpu[..., 0] + 1j * e_gpu[..., 1]
        assert np.abs(e_ref).max() > 1e-4
        assert np.abs(e_gpu - e_ref).max() < 1e-10 * max(1.0, np.abs(e_ref).max())
    finally:
        thc.thc_dyson_destroy(d)


def test_cdiis_loop_matches_oracle_cdiis_loop():
    from paper_2404_17744_gb300 import scf, thc
    case = synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)
    g = grid_for(100.0, 10.0)
    ref = so.run_loop(case, g, 8.0, tol=1e-10, mix="cdiis")
    L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64, mixing="cdiis")
    try:
        conv = L.run(tol=1e-10, max_iter=80)
        recs = L.records
    finally:
        L.close()
    plain = so.run_loop(case, g, 8.0, tol=1e-10)
    print(f"CDIIS: oracle E {ref['E']:.12f} ({ref['iters']} it), GPU E {recs[-1].E:.12f} ({len(recs)} it); "
          f"residual DIIS {plain['iters']} it")
    assert conv and ref["converged"]
    assert abs(recs[-1].E - ref["E"]) < 1e-9 and abs(recs[-1].E - plain["E"]) < 1e-9
    assert abs(len(recs) - ref["iters"]) <= 2


def test_gwsox_loop_matches_oracle_loop():
    """scGWSOX: the loop with the screened direct term (THC_GW | THC_SOX, FP64) against the
    oracle's loop with sigma_gw_thc + SOX, on the same IR grid and bosonic transforms."""
    from paper_2404_17744_gb300 import scf, thc
    case = synth.make_sigma_case(20, 60, 4, 100.0, 17745, identity_S=False, n_occ=8)
    g = grid_for(100.0, 10.0)
    bt = ir.make_bosonic_transforms(g)
    U = o.thc_U(case.X, case.V)

    def sigma_fn(G_tau):
        nt = G_tau.shape[0]
        Gb = G_tau[::-1]
        sox = np.stack([o.sigma_sox_thc(case.X, U, G_tau[k], o.g_minus_tau(Gb[k])) for k in range(nt)])
        return o.sigma_gw_thc(case.X, case.V, G_tau, Gb, bt.to_iw, bt.to_tau) + sox

    ref = so.run_loop(case, g, 8.0, tol=1e-10, sigma_fn=sigma_fn)
    L = scf.GF2Loop(case.X, case.V, case.F, case.S, g, 8.0, precision=thc.THC_FP64, bosonic=bt)
    try:
        conv = L.run(tol=1e-10, max_iter=80)
        recs = L.records
    finally:
        L.close()
    gf2 = so.run_loop(case, g, 8.0, tol=1e-10)
    print(f"scGWSOX oracle E {ref['E']:.12f} ({ref['iters']} it), GPU {recs[-1].E:.12f} ({len(recs)} it); "
          f"GF2 E {gf2['E']:.12f}")
    print("first energies, oracle / GPU:", [f"{h['E']:.10f}" for h in ref["history"][:6]],
          [f"{r.E:.10f}" for r in recs[:6]])
    assert conv and ref["converged"]
    assert abs(recs[-1].E - ref["E"]) < 1e-9
    assert abs(ref["E"] - gf2["E"]) > 1e-7           # the screening changes the converged energy
    for r, h in zip(recs[:4], ref["history"][:4]):
        assert abs(r.E - h["E"]) < 1e-9
