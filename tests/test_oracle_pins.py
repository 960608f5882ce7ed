"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* four-index definitions (brute force on tiny inputs, generic non-symmetric G)
* the one-orbital closed form
* the finite-temperature MP2 closed form of E_dyn[G0] (analytic tau integral)
* the zero-temperature textbook closed-shell MP2 energy (E_dyn[G0] -> 2 E_MP2)
* Sigma_ij = Sigma_ji, Sigma ~ lambda^2 under V -> lambda V, fragment separability
  (appendix of arXiv:2404.17744), and G(0+) + G(beta-) = -S^{-1}
Planted-mistake tests show that a sign or index error in the oracle fails a pin.
"""
import functools

import numpy as np
import pytest
import scipy.linalg

from oracle import thc_oracle as o
from workloads import synth


def _tiny(n, N, seed, n_tau=2, symmetric=False):
    rng = synth.rng_for(seed)
    X = synth.draw_X(n, N, rng)
    V = synth.draw_V(N, rng)
    if symmetric:
        Gt = synth.random_symmetric(n_tau, n, rng)
        Gb = synth.random_symmetric(n_tau, n, rng)
    else:
        Gt = rng.standard_normal((n_tau, n, n))
        Gb = rng.standard_normal((n_tau, n, n))
    return X, V, Gt, Gb


@pytest.mark.parametrize("n,N,seed", [(3, 5, 1), (5, 9, 2), (6, 11, 3)])
def test_sox_thc_equals_four_index(n, N, seed):
    X, V, Gt, Gb = _tiny(n, N, seed)
    v = o.eri_from_thc(X, V)
    ref = o.sigma_four_index(v, Gt, Gb, "sox")
    got = o.sigma_thc(X, V, Gt, Gb, terms="sox")
    assert np.abs(ref).max() > 1e-3
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("n,N,seed", [(3, 5, 4), (5, 9, 5), (6, 11, 6)])
def test_direct_thc_equals_four_index(n, N, seed):
    X, V, Gt, Gb = _tiny(n, N, seed)
    v = o.eri_from_thc(X, V)
    ref = o.sigma_four_index(v, Gt, Gb, "direct")
    got = o.sigma_thc(X, V, Gt, Gb, terms="direct")
    assert np.abs(ref).max() > 1e-3
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_eri_and_U_against_loops():
    n, N = 3, 4
    rng = synth.rng_for(7)
    X = synth.draw_X(n, N, rng)
    V = synth.draw_V(N, rng)
    v = o.eri_from_thc(X, V)
    U = o.thc_U(X, V)
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    acc = 0.0
                    for P in range(N):
                        for Q in range(N):
                            acc += X[p, P] * X[q, P] * V[P, Q] * X[r, Q] * X[s, Q]
                    assert abs(acc - v[p, q, r, s]) < 1e-14
    for P in range(N):
        for q in range(n):
            for s in range(n):
                acc = sum(V[P, Q] * X[q, Q] * X[s, Q] for Q in range(N))
                assert abs(acc - U[P, q, s]) < 1e-14
    # (pq|rs) = sum_P X_pP X_qP U_Prs
    np.testing.assert_allclose(np.einsum("pP,qP,Prs->pqrs", X, X, U), v, atol=1e-14)


@pytest.mark.parametrize("e", [0.7, -0.4, 1e-9])
def test_one_orbital_closed_form(e):
    beta = 20.0
    rng = synth.rng_for(8)
    N = 3
    X = rng.standard_normal((1, N))
    V = synth.draw_V(N, rng)
    vv = float(o.eri_from_thc(X, V)[0, 0, 0, 0])
    tau = np.array([0.3, 2.0, 9.5, 17.0])
    G = o.g0_tau(np.array([[e]]), np.eye(1), 0.0, beta, tau)
    Gb = o.g0_tau(np.array([[e]]), np.eye(1), 0.0, beta, beta - tau)
    d_ref, x_ref = o.one_orbital_sigma(vv, e, beta, tau)
    d = o.sigma_thc(X, V, G, Gb, terms="direct")[:, 0, 0]
    x = o.sigma_thc(X, V, G, Gb, terms="sox")[:, 0, 0]
    np.testing.assert_allclose(d, d_ref, rtol=1e-10)
    np.testing.assert_allclose(x, x_ref, rtol=1e-10)
    # closed form stated directly: Sigma^x = v^2 (1-n)^2 n e^{-e tau}, n = 1/(1+e^{beta e})
    nocc = 1.0 / (1.0 + np.exp(beta * e))
    np.testing.assert_allclose(x, vv ** 2 * (1 - nocc) ** 2 * nocc * np.exp(-e * tau), rtol=1e-10)
    np.testing.assert_allclose(d, -2 * x, rtol=1e-12)


def _mp2_setup(beta, n=4, N=8, n_occ=2, seed=3, identity_S=False):
    case = synth.make_sigma_case(n, N, 4, beta, seed, n_occ=n_occ, identity_S=identity_S)
    tau, w = o.composite_gauss_legendre(beta)
    G = o.g0_tau(case.F, case.S, 0.0, beta, tau)
    Gb = G[::-1]
    v = o.eri_from_thc(case.X, case.V)
    eps, C = scipy.linalg.eigh(case.F, case.S)
    vmo = o.mo_eri(v, C)
    return case, tau, w, G, Gb, v, eps, vmo


@pytest.mark.parametrize("beta", [5.0, 20.0])
def test_energy_matches_finite_T_closed_form(beta):
    case, tau, w, G, Gb, v, eps, vmo = _mp2_setup(beta)
    Sd = o.sigma_four_index(v, G, Gb, "direct")
    Sx = o.sigma_four_index(v, G, Gb, "sox")
    Ed = o.energy_dyn_tau(Gb, Sd, w)
    Ex = o.energy_dyn_tau(Gb, Sx, w)
    cd, cx = o.mp2_finite_T(vmo, eps, beta)
    assert abs(Ed - cd) < 1e-12 * abs(cd)
    assert abs(Ex - cx) < 1e-12 * abs(cx)
    assert Ed < 0 < Ex


def test_energy_zero_temperature_is_twice_textbook_mp2():
    beta = 400.0
    case, tau, w, G, Gb, v, eps, vmo = _mp2_setup(beta)
    S = o.sigma_thc(case.X, case.V, G, Gb)
    E = o.energy_dyn_tau(Gb, S, w)
    emp2 = o.mp2_zero_T_closed_shell(vmo, eps, 2)
    assert abs(E - 2 * emp2) < 1e-12 * abs(emp2)


def test_symmetry_and_V_scaling():
    case = synth.make_sigma_case(6, 14, 6, 30.0, 11)
    S1 = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt)
    np.testing.assert_allclose(S1, np.swapaxes(S1, 1, 2), atol=1e-15 * np.abs(S1).max())
    S2 = o.sigma_thc(case.X, 1.7 * case.V, case.G_tau, case.G_bmt)
    np.testing.assert_allclose(S2, 1.7 ** 2 * S1, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", [3, 4])
def test_sox_intermediate_D_is_symmetric(seed):
    """D_PR = sum_{v w q s} G_Pw U_Rvw G_Rq U_Pqs G_vs(-tau) is symmetric in (P, R) when
    G(tau) and G(-tau) are (rename w <-> q, v <-> s and use U_Pqs = U_Psq); the GPU paths
    compute D on and above the diagonal only and mirror it.  A non-symmetric G breaks it."""
    case = synth.make_sigma_case(11, 37, 4, 30.0, seed, identity_S=False, n_occ=4)
    U = o.thc_U(case.X, case.V)
    for k in range(case.n_tau):
        G, Gm = case.G_tau[k], o.g_minus_tau(case.G_bmt[k])
        _, it = o.sigma_sox_thc(case.X, U, G, Gm, return_intermediates=True)
        D = it["D"]
        assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    rng = np.random.default_rng(seed)
    Gn = G + 0.1 * np.abs(G).max() * rng.standard_normal(G.shape)
    _, it = o.sigma_sox_thc(case.X, U, Gn, Gm, return_intermediates=True)
    assert np.abs(it["D"] - it["D"].T).max() > 1e-6 * np.abs(it["D"]).max()


def test_fragment_separability():
    """Two non-interacting fragments (appendix): block-diagonal Sigma, additive E_dyn."""
    beta = 15.0
    a = synth.make_sigma_case(3, 5, 8, beta, 21, n_occ=1)
    b = synth.make_sigma_case(4, 7, 8, beta, 22, n_occ=2)
    X = scipy.linalg.block_diag(a.X, b.X)
    V = scipy.linalg.block_diag(a.V, b.V)
    F = scipy.linalg.block_diag(a.F, b.F)
    tau, w = o.composite_gauss_legendre(beta, n_panels_per_side=12, order=16)
    G = o.g0_tau(F, np.eye(7), 0.0, beta, tau)
    Gb = G[::-1]
    S = o.sigma_thc(X, V, G, Gb)
    assert np.abs(S[:, :3, 3:]).max() < 1e-15
    Ga = o.g0_tau(a.F, np.eye(3), 0.0, beta, tau)
    Gbb = o.g0_tau(b.F, np.eye(4), 0.0, beta, tau)
    Sa = o.sigma_thc(a.X, a.V, Ga, Ga[::-1])
    Sb = o.sigma_thc(b.X, b.V, Gbb, Gbb[::-1])
    np.testing.assert_allclose(S[:, :3, :3], Sa, atol=1e-14)
    np.testing.assert_allclose(S[:, 3:, 3:], Sb, atol=1e-14)
    E = o.energy_dyn_tau(Gb, S, w)
    Ea = o.energy_dyn_tau(Ga[::-1], Sa, w)
    Eb = o.energy_dyn_tau(Gbb[::-1], Sb, w)
    assert abs(E - (Ea + Eb)) < 1e-13


def test_g0_boundary_identity_and_generator_agreement():
    case = synth.make_sigma_case(7, 10, 6, 50.0, 31, identity_S=False, n_occ=3)
    G = o.g0_tau(case.F, case.S, 0.0, case.beta, np.array([0.0, case.beta]))
    np.testing.assert_allclose(G[0] + G[1], -np.linalg.inv(case.S), atol=1e-13)
    # particle number per spin: gamma = -G(beta^-), Tr[gamma S] = sum_k 1/(1 + e^{beta eps_k})
    n_exact = np.sum(1.0 / (1.0 + np.exp(case.beta * case.eps)))
    assert abs(np.trace(-G[1] @ case.S) - n_exact) < 1e-12
    assert abs(n_exact - 3.0) < 1e-2
    G_or = o.g0_tau(case.F, case.S, 0.0, case.beta, case.tau)
    np.testing.assert_allclose(G_or, case.G_tau, atol=1e-13)


# ------------------------------------------------------------ planted mistakes
def test_planted_sign_mistake_fails_mp2_pin(monkeypatch):
    monkeypatch.setattr(o, "C_SOX", -1.0)
    beta = 400.0
    case, tau, w, G, Gb, v, eps, vmo = _mp2_setup(beta)
    E = o.energy_dyn_tau(Gb, o.sigma_thc(case.X, case.V, G, Gb), w)
    emp2 = o.mp2_zero_T_closed_shell(vmo, eps, 2)
    assert abs(E - 2 * emp2) > 1e-3 * abs(emp2)


def test_planted_index_mistake_fails_four_index_pin(monkeypatch):
    X, V, Gt, Gb = _tiny(5, 9, 2)
    v = o.eri_from_thc(X, V)
    ref = o.sigma_four_index(v, Gt, Gb, "sox")
    real = o.sigma_sox_thc

    def wrong(X, U, G, Gm, return_intermediates=False):
        return real(X, U, G.T, Gm)          # G_Rq built from G^T: a transposed operand

    monkeypatch.setattr(o, "sigma_sox_thc", wrong)
    got = o.sigma_thc(X, V, Gt, Gb, terms="sox")
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()


def test_planted_dropped_term_fails_closed_form(monkeypatch):
    """Dropping the polarisation's G(-tau) factor (a lost term) breaks the MP2 pin."""
    def wrong(X, V, G, Gm):
        GX = X.T @ G @ X
        W = V @ GX @ V
        return o.C_DIRECT * (X @ (GX * W) @ X.T)

    monkeypatch.setattr(o, "sigma_direct_thc", wrong)
    beta = 20.0
    case, tau, w, G, Gb, v, eps, vmo = _mp2_setup(beta)
    Ed = o.energy_dyn_tau(Gb, o.sigma_thc(case.X, case.V, G, Gb, terms="direct"), w)
    cd, _ = o.mp2_finite_T(vmo, eps, beta)
    assert abs(Ed - cd) > 1e-3 * abs(cd)


def test_golden_thc20_regression():
    """The oracle reproduces the stored thc20 values (written by tests/golden/make_golden.py)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "thc20_oracle.json")
    g = json.load(open(path))
    case = synth.make_workload("thc20")
    Sd = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt, terms="direct")
    Sx = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt, terms="sox")
    assert abs(o.energy_dyn_tau(case.G_bmt, Sd, case.tau_w) - g["E_dyn_direct"]) < 1e-13
    assert abs(o.energy_dyn_tau(case.G_bmt, Sx, case.tau_w) - g["E_dyn_sox"]) < 1e-13
    for k, i, j, d, x in g["samples"]:
        assert abs(Sd[k, i, j] - d) < 1e-14 and abs(Sx[k, i, j] - x) < 1e-14


def test_mlp_oracle_gradients_against_finite_differences():
    """Backpropagation of the proposal network's loss equals central differences."""
    from oracle import mlp_oracle as mo
    rng = np.random.default_rng(3)
    B, din, H, dout = 7, 6, 9, 4
    X = rng.standard_normal((B, din))
    T = rng.standard_normal((B, dout))
    W1 = rng.standard_normal((H, din)) * 0.5
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((dout, H)) * 0.5
    b2 = rng.standard_normal(dout) * 0.1
    loss, gW1, gb1, gW2, gb2 = mo.loss_and_grads(X, T, W1, b1, W2, b2)
    h = 1e-6
    for P, G in ((W1, gW1), (b1, gb1), (W2, gW2), (b2, gb2)):
        flat = P.reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 11)):
            old = flat[i]
            flat[i] = old + h
            lp = mo.loss_and_grads(X, T, W1, b1, W2, b2)[0]
            flat[i] = old - h
            lm = mo.loss_and_grads(X, T, W1, b1, W2, b2)[0]
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - G.reshape(-1)[i]) < 1e-7


def test_mlp_oracle_forward_hand_computed():
    """A 2-sample, 3 -> 2 -> 2 network evaluated by hand:
    sample 1: z = (1 - 1 + 0.5, -1 + 2 - 1) = (0.5, 0), relu keeps (0.5, 0), y = (2*0.5 + 1, -2) = (2, -2);
    sample 2: z = (3 + 0.5, -1 - 1) = (3.5, -2), relu (3.5, 0), y = (2*3.5 + 1, -2) = (8, -2);
    targets (1, -2), (8, 0): residuals (1, 0), (0, -2), loss (1 + 4) / 4 = 1.25."""
    from oracle import mlp_oracle as mo
    X = np.array([[1.0, 2.0, -1.0], [0.0, -1.0, 3.0]])
    W1 = np.array([[1.0, 0.0, 1.0], [-1.0, 1.0, 0.0]])
    b1 = np.array([0.5, -1.0])
    W2 = np.array([[2.0, -1.0], [0.0, 3.0]])
    b2 = np.array([1.0, -2.0])
    T = np.array([[1.0, -2.0], [8.0, 0.0]])
    for fp16 in (False, True):   # every weight is exact in FP16
        Y, _ = mo.forward(X, W1, b1, W2, b2, fp16_weights=fp16)
        assert np.array_equal(Y, np.array([[2.0, -2.0], [8.0, -2.0]]))
        loss, gW1, gb1, gW2, gb2 = mo.loss_and_grads(X, T, W1, b1, W2, b2, fp16_weights=fp16)
        assert loss == 1.25
        # dL/dy = 2 r / 4 = ((0.5, 0), (0, -1)); dL/db2 = column sums
        assert np.array_equal(gb2, np.array([0.5, -1.0]))
        # dL/dW2 = dY^T A1 with A1 = ((0.5, 0), (3.5, 0))
        assert np.array_equal(gW2, np.array([[0.25, 0.0], [-3.5, 0.0]]))
        # hidden unit 2 is inactive in both samples (z <= 0): no gradient reaches W1[1], b1[1]
        assert np.array_equal(gW1[1], np.zeros(3)) and gb1[1] == 0.0
        # unit 1: dz = dY @ W2[:, 0] = (0.5*2 + 0, 0 + (-1)*0) = (1, 0) -> gW1[0] = x_1, gb1[0] = 1
        assert np.array_equal(gW1[0], X[0]) and gb1[0] == 1.0


@pytest.mark.parametrize("rows", [1, 7, 64])
def test_sox_rowwise_equals_scheme(rows):
    """sigma_sox_thc_rows (D formed a slice of P at a time, for the full-size golden values)
    evaluates the same steps as sigma_sox_thc, on ragged slices too."""
    case = synth.make_sigma_case(11, 45, 3, 20.0, 31)
    U = o.thc_U(case.X, case.V)
    for k in range(case.n_tau):
        G, Gm = case.G_tau[k], o.g_minus_tau(case.G_bmt[k])
        a = o.sigma_sox_thc(case.X, U, G, Gm)
        b = o.sigma_sox_thc_rows(case.X, U, G, Gm, rows=rows)
        assert np.abs(a - b).max() <= 1e-15 * np.abs(a).max()


@pytest.mark.parametrize("n,N,seed", [(3, 7, 1), (4, 9, 2)])
def test_uhf_thc_equals_spin_orbital_definition(n, N, seed):
    """The unrestricted THC route equals the spin-orbital four-index definition for two
    different (non-symmetric) spin Green's functions."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, N)) / np.sqrt(n)
    V = synth.draw_V(N, rng)
    v = o.eri_from_thc(X, V)
    U = o.thc_U(X, V)
    Ga, Gb, Gma, Gmb = (rng.standard_normal((n, n)) for _ in range(4))
    Sa, Sb = o.sigma_uhf_thc(X, V, U, Ga, Gb, Gma, Gmb)
    Ra, Rb = o.sigma_uhf_spin_orbital(v, Ga, Gb, Gma, Gmb)
    scale = max(np.abs(Ra).max(), np.abs(Rb).max())
    assert np.abs(Sa - Ra).max() <= 1e-13 * scale and np.abs(Sb - Rb).max() <= 1e-13 * scale
    # exchanging the spins exchanges the self-energies
    Tb, Ta = o.sigma_uhf_thc(X, V, U, Gb, Ga, Gmb, Gma)
    assert np.abs(Ta - Sa).max() <= 1e-13 * scale and np.abs(Tb - Sb).max() <= 1e-13 * scale


def test_uhf_reduces_to_restricted_for_equal_spins():
    """With G_alpha = G_beta both spin self-energies equal the restricted (per-spin) one,
    and the unrestricted energy equals the restricted energy; with unequal spins the
    bubble of one spin feels the other."""
    case = synth.make_sigma_case(7, 19, 4, 30.0, 12, n_occ=3)
    U = o.thc_U(case.X, case.V)
    R = o.sigma_thc(case.X, case.V, case.G_tau, case.G_bmt)
    Sa = np.empty_like(R)
    Sb = np.empty_like(R)
    for k in range(case.n_tau):
        G, Gm = case.G_tau[k], o.g_minus_tau(case.G_bmt[k])
        Sa[k], Sb[k] = o.sigma_uhf_thc(case.X, case.V, U, G, G, Gm, Gm)
    scale = np.abs(R).max()
    assert np.abs(Sa - R).max() <= 1e-13 * scale and np.abs(Sb - R).max() <= 1e-13 * scale
    E_r = o.energy_dyn_tau(case.G_bmt, R, case.tau_w)
    assert abs(o.energy_dyn_tau_uhf(case.G_bmt, case.G_bmt, Sa, Sb, case.tau_w) - E_r) <= 1e-13 * abs(E_r)
    # a beta spin with one electron fewer (mu between the second and third levels) changes
    # the alpha self-energy through the bubble
    Gb_tau = synth.noninteracting_G(case.F, case.S, 0.5 * (case.eps[1] + case.eps[2]), case.beta, case.tau)
    G, Gm = case.G_tau[0], o.g_minus_tau(case.G_bmt[0])
    Sa2, _ = o.sigma_uhf_thc(case.X, case.V, U, G, Gb_tau[0], Gm, o.g_minus_tau(Gb_tau[-1]))
    assert np.abs(Sa2 - Sa[0]).max() > 1e-6 * scale


@functools.lru_cache(maxsize=None)
def _bosonic(beta, wmax=10.0):
    from workloads import ir
    g = ir.make_loop_grid(beta, wmax)
    return g, ir.make_bosonic_transforms(g)


def test_gw_weak_coupling_is_the_second_order_direct_term():
    """Sigma^GW(lambda V) / lambda^2 tends to the second-order direct term as lambda -> 0,
    with a remainder linear in lambda (the first screening correction)."""
    g, bt = _bosonic(50.0)
    case = synth.make_sigma_case(6, 14, 4, 50.0, 31, identity_S=False, n_occ=3)
    G = synth.noninteracting_G(case.F, case.S, 0.0, 50.0, g.tau)
    Gb = G[::-1]
    ref = o.sigma_thc(case.X, case.V, G, Gb, terms="direct")
    d = []
    for lam in (1e-2, 5e-3):
        S = o.sigma_gw_thc(case.X, lam * case.V, G, Gb, bt.to_iw, bt.to_tau) / lam ** 2
        d.append(np.abs(S - ref).max() / np.abs(ref).max())
    assert d[0] < 5e-2 and 1.6 < d[0] / d[1] < 2.4    # remainder ~ lambda


def test_gw_one_orbital_closed_form():
    """One orbital, one THC point: Pi~ is constant in tau, so only Omega = 0 screens:
    Sigma^GW(tau) = Sigma^(2)(tau) / (1 + 2 v beta n (1 - n)), v = V X^4."""
    beta = 50.0
    g, bt = _bosonic(beta)
    x, V, e = 0.9, 0.7, 0.03   # beta e = 1.5: n (1 - n) ~ 0.15, so screening is strong
    X = np.array([[x]])
    Vm = np.array([[V]])
    G = np.array([[[o.fermi_pair(np.array([e]), beta)[1][0] * -np.exp(-e * t)]] for t in g.tau])
    Gb = G[::-1].copy()
    S = o.sigma_gw_thc(X, Vm, G, Gb, bt.to_iw, bt.to_tau)[:, 0, 0]
    n_occ, n_vir = o.fermi_pair(np.array([e]), beta)
    v = V * x ** 4
    s2, _ = o.one_orbital_sigma(v, e, beta, g.tau)
    expect = s2 / (1.0 + 2.0 * v * beta * n_occ[0] * n_vir[0])
    assert np.abs(S - expect).max() <= 1e-9 * np.abs(expect).max()
    assert np.abs(expect - s2).max() > 1e-3 * np.abs(s2).max()   # screening is not negligible here


def test_gw_symmetric():
    g, bt = _bosonic(50.0)
    case = synth.make_sigma_case(7, 20, 4, 50.0, 12, n_occ=3)
    G = synth.noninteracting_G(case.F, case.S, 0.0, 50.0, g.tau)
    S = o.sigma_gw_thc(case.X, case.V, G, G[::-1], bt.to_iw, bt.to_tau)
    assert np.abs(S - np.swapaxes(S, 1, 2)).max() <= 1e-13 * np.abs(S).max()


def _uhf_pair(case, g):
    """Two different spin blocks: G_a of F, G_b of F shifted by a symmetric perturbation."""
    rng = np.random.default_rng(77)
    Fb = case.F + 0.2 * synth.random_symmetric(1, case.n, rng)[0]
    Ga = synth.noninteracting_G(case.F, case.S, 0.0, g.basis.beta, g.tau)
    Gb = synth.noninteracting_G(Fb, case.S, 0.0, g.basis.beta, g.tau)
    return Ga, Gb


def test_gw_uhf_equal_spins_is_the_restricted_term():
    g, bt = _bosonic(50.0)
    case = synth.make_sigma_case(7, 20, 4, 50.0, 13, identity_S=False, n_occ=3)
    G = synth.noninteracting_G(case.F, case.S, 0.0, 50.0, g.tau)
    Sa, Sb = o.sigma_gw_uhf_thc(case.X, case.V, G, G[::-1], G, G[::-1], bt.to_iw, bt.to_tau)
    R = o.sigma_gw_thc(case.X, case.V, G, G[::-1], bt.to_iw, bt.to_tau)
    scale = np.abs(R).max()
    assert np.abs(Sa - R).max() <= 1e-13 * scale and np.abs(Sb - R).max() <= 1e-13 * scale


def test_gw_uhf_weak_coupling_is_the_unrestricted_bubble():
    """Sigma^GW_s(lambda V) / lambda^2 tends to the direct term of sigma_uhf_thc (pinned to
    the spin-orbital definition) with a remainder linear in lambda; the spins differ."""
    g, bt = _bosonic(50.0)
    case = synth.make_sigma_case(6, 14, 4, 50.0, 31, identity_S=False, n_occ=3)
    Ga, Gb = _uhf_pair(case, g)
    nt = len(g.tau)
    U = o.thc_U(case.X, case.V)
    ref = [np.empty_like(Ga), np.empty_like(Gb)]
    for k in range(nt):
        Gma, Gmb = o.g_minus_tau(Ga[nt - 1 - k]), o.g_minus_tau(Gb[nt - 1 - k])
        ta, tb = o.sigma_uhf_thc(case.X, case.V, U, Ga[k], Gb[k], Gma, Gmb)
        ref[0][k] = ta - o.sigma_sox_thc(case.X, U, Ga[k], Gma)
        ref[1][k] = tb - o.sigma_sox_thc(case.X, U, Gb[k], Gmb)
    assert np.abs(ref[0] - ref[1]).max() > 1e-3 * np.abs(ref[0]).max()   # the spins really differ
    for s in range(2):
        d = []
        for lam in (1e-2, 5e-3):
            S = o.sigma_gw_uhf_thc(case.X, lam * case.V, Ga, Ga[::-1], Gb, Gb[::-1], bt.to_iw, bt.to_tau)[s]
            d.append(np.abs(S / lam ** 2 - ref[s]).max() / np.abs(ref[s]).max())
        assert d[0] < 5e-2 and 1.6 < d[0] / d[1] < 2.4, (s, d)


def test_gw_uhf_one_orbital_closed_form():
    """One orbital, one THC point, levels e_a != e_b: each spin's bubble G_s(tau) G_s(-tau)
    = -n_s (1 - n_s) is constant in tau, so only Omega = 0 screens, by the sum over both
    spins: Sigma^GW_s(tau) = -v^2 c (1 - n_s) e^{-e_s tau} / (1 + v beta c) with
    c = n_a (1 - n_a) + n_b (1 - n_b) and v = V X^4."""
    beta = 50.0
    g, bt = _bosonic(beta)
    x, V, ea, eb = 0.9, 0.7, 0.03, -0.02
    X = np.array([[x]])
    Vm = np.array([[V]])

    def G_of(e):
        nv = o.fermi_pair(np.array([e]), beta)[1][0]
        return np.array([[[-nv * np.exp(-e * t)]] for t in g.tau])
    Ga, Gb = G_of(ea), G_of(eb)
    Sa, Sb = o.sigma_gw_uhf_thc(X, Vm, Ga, Ga[::-1].copy(), Gb, Gb[::-1].copy(), bt.to_iw, bt.to_tau)
    na, nva = (v[0] for v in o.fermi_pair(np.array([ea]), beta))
    nb, nvb = (v[0] for v in o.fermi_pair(np.array([eb]), beta))
    c = na * nva + nb * nvb
    v = V * x ** 4
    for S, nv, e in ((Sa, nva, ea), (Sb, nvb, eb)):
        expect = -v * v * c * nv * np.exp(-e * g.tau) / (1.0 + v * beta * c)
        assert np.abs(S[:, 0, 0] - expect).max() <= 1e-9 * np.abs(expect).max()
