"""Pins of the IR basis (an input built in workloads.ir) and of the oracle's
self-consistent loop (oracle/scf_oracle.py), against facts that do not come
from the code under test:

* single-pole functions: G(tau) = -e^{-e tau}/(1 + e^{-beta e}) has the exact
  transform 1/(i w_n - e); the basis must reproduce both;
* Dyson with Sigma = 0 gives the analytic noninteracting G; G(0+) + G(beta-) = -S^{-1};
* the IR-coefficient energy of Sigma[G0] at G0 equals the finite-temperature
  MP2 closed form; the Matsubara-sum route (Eq. E2b) equals the tau route;
* the converged loop energy does not depend on the mixing scheme, and the
  electron count is conserved.
"""
import functools

import numpy as np
import pytest
import scipy.linalg

from oracle import scf_oracle as so
from oracle import thc_oracle as o
from workloads import ir, synth


@functools.lru_cache(maxsize=None)
def grid_for(beta, wmax):
    return ir.make_loop_grid(beta, wmax)


def _pole(e, beta, tau):
    if e >= 0:
        return -np.exp(-e * tau) / (1 + np.exp(-beta * e))
    return -np.exp(e * (beta - tau)) / (1 + np.exp(beta * e))


@pytest.mark.parametrize("beta,wmax", [(50.0, 10.0), (100.0, 10.0), (1000.0, 100.0)])
def test_ir_basis_single_poles(beta, wmax):
    g = grid_for(beta, wmax)
    assert len(g.tau) == g.basis.L and len(g.iw) >= g.basis.L
    assert np.abs(g.tau + g.tau[::-1] - beta).max() < 1e-12 * beta
    assert np.abs(g.iw + g.iw[::-1]).max() < 1e-12
    # the sampling matrices stay well conditioned (the Matsubara one grows slowly with Lambda)
    assert np.linalg.cond(g.U_tau) < 1e3 and np.linalg.cond(g.U_iw) < 3e3
    for e in (-1.9, -0.2, 0.0, 0.4, 2.5):
        gl = g.fit_tau @ _pole(e, beta, g.tau)
        assert np.abs(g.U_iw @ gl - 1.0 / (1j * g.iw - e)).max() < 1e-8
        tt = np.array([0.0, 0.1, beta / 3, beta - 0.05, beta])
        assert np.abs(g.basis.u(tt).T @ gl - _pole(e, beta, tt)).max() < 1e-8
        back = (g.U_tau @ (g.fit_iw @ (1.0 / (1j * g.iw - e)))).real
        assert np.abs(back - _pole(e, beta, g.tau)).max() < 1e-8


def _case(beta=50.0):
    return synth.make_sigma_case(6, 14, 4, beta, 31, identity_S=False, n_occ=3)


def _sigma_at(case, G):
    U = o.thc_U(case.X, case.V)
    nt = G.shape[0]
    return np.stack([o.sigma_sox_thc(case.X, U, G[k], -G[nt - 1 - k]) +
                     o.sigma_direct_thc(case.X, case.V, G[k], -G[nt - 1 - k]) for k in range(nt)])


def test_dyson_noninteracting_and_boundary_identity():
    case = _case()
    g = grid_for(50.0, 10.0)
    G, mu = so.solve_dyson(g, case.S, case.F, None, 3.0, 0.0)
    # the count is exact at the returned mu, and mu sits in the gap
    n_exact = np.sum(1.0 / (1.0 + np.exp(50.0 * (case.eps - mu))))
    assert abs(n_exact - 3.0) < 2e-8
    assert np.abs(G - o.g0_tau(case.F, case.S, mu, 50.0, g.tau)).max() < 5e-9
    gl = g.fit_tau @ G.reshape(len(g.tau), -1)
    G0p, Gbm = (g.u_zero @ gl).reshape(6, 6), (g.u_beta @ gl).reshape(6, 6)
    assert np.abs(G0p + Gbm + np.linalg.inv(case.S)).max() < 5e-9


def test_ir_energy_matches_finite_T_mp2_and_matsubara_route():
    case = _case()
    g = grid_for(50.0, 10.0)
    G, mu = so.solve_dyson(g, case.S, case.F, None, 3.0, 0.0)
    Sig = _sigma_at(case, G)
    E_ir = so.energy_ir(g, G, Sig)
    eps, C = scipy.linalg.eigh(case.F, case.S)
    cd, cx = o.mp2_finite_T(o.mo_eri(o.eri_from_thc(case.X, case.V), C), eps - mu, 50.0)
    assert abs(E_ir - (cd + cx)) < 1e-11
    assert abs(so.energy_matsubara(g, G, Sig, n_max=4000) - E_ir) < 5e-9


def test_loop_converged_energy_independent_of_mixing():
    case = _case()
    g = grid_for(50.0, 10.0)
    r1 = so.run_loop(case, g, 3.0, tol=1e-11)
    r2 = so.run_loop(case, g, 3.0, tol=1e-11, damping=0.7, n_damp=4, diis_size=4)
    assert r1["converged"] and r2["converged"]
    assert abs(r1["E"] - r2["E"]) < 1e-9
    for h in r1["history"]:
        assert abs(h["n"] - 3.0) < 1e-9
    assert np.abs(r1["Sigma"] - np.swapaxes(r1["Sigma"], 1, 2)).max() < 1e-12
    # the self-consistent energy differs from the first (one-shot) one: the loop did work
    assert abs(r1["history"][0]["E"] - r1["E"]) > 1e-4


def test_planted_wrong_parity_fails_energy_pin(monkeypatch):
    case = _case()
    g = grid_for(50.0, 10.0)
    G, mu = so.solve_dyson(g, case.S, case.F, None, 3.0, 0.0)
    Sig = _sigma_at(case, G)
    eps, C = scipy.linalg.eigh(case.F, case.S)
    cd, cx = o.mp2_finite_T(o.mo_eri(o.eri_from_thc(case.X, case.V), C), eps - mu, 50.0)
    monkeypatch.setattr(so, "parity", lambda grid: np.ones(grid.basis.L))
    assert abs(so.energy_ir(g, G, Sig) - (cd + cx)) > 1e-6


def test_count_slope_matches_finite_difference():
    """dN/dmu from dG/dmu = -G S G equals a central difference of the count."""
    case = _case()
    g = grid_for(50.0, 10.0)
    G, mu = so.solve_dyson(g, case.S, case.F, None, 3.0, 0.0)
    Sig = _sigma_at(case, G)
    Siw = so.sigma_iw(g, Sig)
    for m in (mu, mu + 0.3):
        h = 1e-5
        fd = (so.electron_count(g, case.S, so.dyson_iw(g, case.S, case.F, Siw, m + h))
              - so.electron_count(g, case.S, so.dyson_iw(g, case.S, case.F, Siw, m - h))) / (2 * h)
        an = so.electron_count_slope(g, case.S, so.dyson_iw(g, case.S, case.F, Siw, m))
        assert an > 0 and abs(an - fd) < 1e-6 * max(1.0, abs(an))


def test_commutator_residual_vanishes_at_fixed_points():
    """e = H G S - S G H is zero for the noninteracting G with Sigma = 0 and for the
    converged loop, and clearly non-zero for an unconverged pair."""
    case = _case()
    g = grid_for(50.0, 10.0)
    G0, mu0, G0iw = so.solve_dyson(g, case.S, case.F, None, 3.0, 0.0, return_iw=True)
    e0 = so.commutator_residual(g, case.S, case.F, G0iw, np.zeros_like(G0))
    assert np.abs(e0).max() < 1e-12
    Sig = _sigma_at(case, G0)                 # Sigma[G0] with G0: not self-consistent
    assert np.abs(so.commutator_residual(g, case.S, case.F, G0iw, Sig)).max() > 1e-4
    r = so.run_loop(case, g, 3.0, tol=1e-12)
    G, mu, Giw = so.solve_dyson(g, case.S, case.F, r["Sigma"], 3.0, r["mu"], return_iw=True)
    assert np.abs(so.commutator_residual(g, case.S, case.F, Giw, r["Sigma"])).max() < 1e-7


def test_cdiis_reaches_the_diis_fixed_point():
    case = _case()
    g = grid_for(50.0, 10.0)
    r1 = so.run_loop(case, g, 3.0, tol=1e-11)
    r2 = so.run_loop(case, g, 3.0, tol=1e-11, mix="cdiis")
    assert r1["converged"] and r2["converged"]
    assert abs(r1["E"] - r2["E"]) < 1e-9


def _linear_map(d, seed):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((d, d)))[0]
    A = Q @ np.diag(rng.uniform(-0.8, 0.8, d)) @ Q.T       # a contraction
    b = rng.standard_normal(d)
    x_star = np.linalg.solve(np.eye(d) - A, b)
    return (lambda x: A @ x + b), x_star, rng


def test_diis_is_exact_on_a_linear_map_with_d_plus_one_iterates():
    """Pulay / Anderson property: for f(x) = A x + b in d dimensions, d + 1 affinely
    independent iterates make the residual combination vanish, and the mixed output is
    the fixed point (I - A)^{-1} b."""
    f, x_star, rng = _linear_map(4, 3)
    xs = [rng.standard_normal(4) for _ in range(5)]
    hist = [(f(x), f(x) - x) for x in xs]
    assert np.allclose(so._diis(hist, 6), x_star, atol=1e-12, rtol=0)
    assert np.allclose(so._diis(hist, 5), x_star, atol=1e-12, rtol=0)   # exactly d + 1 pairs
    # a history window shorter than d + 1 does not reach it
    assert np.abs(so._diis(hist, 3) - x_star).max() > 1e-6


@pytest.mark.parametrize("complex_res", [False, True])
def test_diis_two_point_closed_form(complex_res):
    """Two pairs: c minimises |c r1 + (1 - c) r2| over real c, so
    c = -Re<r2, r1 - r2> / |r1 - r2|^2 and the result is c out1 + (1 - c) out2
    (complex residuals enter through their real and imaginary parts alike)."""
    rng = np.random.default_rng(11)
    shape = (3, 5)
    o1, o2 = rng.standard_normal(shape), rng.standard_normal(shape)
    r1, r2 = rng.standard_normal(shape), rng.standard_normal(shape)
    if complex_res:
        r1 = r1 + 1j * rng.standard_normal(shape)
        r2 = r2 + 1j * rng.standard_normal(shape)
    flat = lambda r: np.concatenate([np.real(r).ravel(), np.imag(r).ravel()])  # noqa: E731
    d = flat(r1) - flat(r2)
    c = -(flat(r2) @ d) / (d @ d)
    assert np.allclose(so._diis([(o1, r1), (o2, r2)], 6), c * o1 + (1 - c) * o2, atol=1e-13, rtol=0)
    # the last `size` pairs only
    assert np.allclose(so._diis([(o2 * 7, r1 * 3), (o1, r1), (o2, r2)], 2), c * o1 + (1 - c) * o2,
                       atol=1e-13, rtol=0)
