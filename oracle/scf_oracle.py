"""FP64 CPU oracle of the self-consistent GF2 loop (test infrastructure only).

Follows Sec. II.A of arXiv:2404.17744 with the readings stated in
thc_oracle.py: the Dyson equation in the non-orthogonal AO basis,
    G(i w_n) = [(i w_n + mu) S - F - Sigma(i w_n)]^{-1},
the chemical potential re-optimised at every iteration so that the electron
count Tr[gamma S] (gamma = -G(beta^-), per spin) is fixed (appendix, case 2),
the Galitskii-Migdal dynamical energy (Eq. E2b), and damping followed by
DIIS on the self-energy (Sec. III.A names damping and a frequency-dependent
commutator DIIS; any linear combination of self-energies is allowed,
appendix comment 1).

The tau <-> i w transforms use the IR sparse-sampling matrices of
workloads.ir (an input, like the tau grid); every transform, inverse,
search and sum here is this module's own NumPy code.  It shares no code
with the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize

from oracle import thc_oracle as o


def sigma_iw(grid, Sigma_tau):
    """Sigma(i w_m) = U_iw (fit_tau Sigma(tau)), complex, shape (n_iw, n, n)."""
    n_tau, n, _ = Sigma_tau.shape
    sig_l = grid.fit_tau @ Sigma_tau.reshape(n_tau, n * n)
    return (grid.U_iw @ sig_l).reshape(-1, n, n)


def dyson_iw(grid, S, F, Siw, mu):
    """G(i w_m) = [(i w_m + mu) S - F - Sigma(i w_m)]^{-1} for every sampled w_m."""
    return np.stack([np.linalg.inv((1j * w + mu) * S - F - Siw[m]) for m, w in enumerate(grid.iw)])


def electron_count(grid, S, Giw):
    """Tr[gamma S] per spin, gamma = -G(beta^-) = -sum_l u_l(beta) g_l, g = fit_iw G(i w)."""
    n = S.shape[0]
    g_l = grid.fit_iw @ Giw.reshape(len(grid.iw), n * n)
    G_beta = (grid.u_beta @ g_l).real.reshape(n, n)
    return float(np.trace(-G_beta @ S))


def electron_count_slope(grid, S, Giw):
    """dN/dmu of the count above at fixed Sigma: dG(i w)/dmu = -G S G, so
    dN/dmu = Tr[(d gamma/dmu) S] = sum_l u_l(beta) Tr[(fit_iw (G S G))_l S]."""
    n = S.shape[0]
    GSG = np.stack([g @ S @ g for g in Giw])
    d_l = grid.fit_iw @ GSG.reshape(len(grid.iw), n * n)
    return float(np.trace((grid.u_beta @ d_l).real.reshape(n, n) @ S))


def commutator_residual(grid, S, F, Giw, Sigma_out_tau):
    """Frequency-dependent commutator residual of the self-consistency (CDIIS, Sec. III.A):
    e(i w_m) = H(i w_m) G(i w_m) S - S G(i w_m) H(i w_m) with H = F + Sigma_out(i w_m),
    G the Green's function the self-energy Sigma_out was evaluated from.  At the fixed
    point G^{-1} = (i w + mu) S - H, so H G S = (i w + mu) S G S - S = S G H: e = 0."""
    H = F[None, :, :] + sigma_iw(grid, Sigma_out_tau)
    return np.einsum("wij,wjk,kl->wil", H, Giw, S) - np.einsum("ij,wjk,wkl->wil", S, Giw, H)


def g_tau_from_iw(grid, Giw):
    n = Giw.shape[1]
    g_l = (grid.fit_iw @ Giw.reshape(len(grid.iw), n * n)).real
    return (grid.U_tau @ g_l).reshape(-1, n, n)


def solve_dyson(grid, S, F, Sigma_tau, n_elec, mu0=0.0, tol=1e-12, return_iw=False):
    """(G(tau), mu) with the electron count fixed; Sigma_tau None means Sigma = 0.
    return_iw adds G(i w_m) at the sampled frequencies as a third value."""
    n = S.shape[0]
    Siw = np.zeros((len(grid.iw), n, n), dtype=complex) if Sigma_tau is None else sigma_iw(grid, Sigma_tau)

    def count(mu):
        return electron_count(grid, S, dyson_iw(grid, S, F, Siw, mu)) - n_elec

    a, b = mu0 - 0.25, mu0 + 0.25
    fa, fb = count(a), count(b)
    step = 0.5
    while fa > 0:
        a -= step
        step *= 2
        fa = count(a)
    step = 0.5
    while fb < 0:
        b += step
        step *= 2
        fb = count(b)
    mu = scipy.optimize.brentq(count, a, b, xtol=1e-15, rtol=1e-15, maxiter=200)
    Giw = dyson_iw(grid, S, F, Siw, mu)
    if return_iw:
        return g_tau_from_iw(grid, Giw), mu, Giw
    return g_tau_from_iw(grid, Giw), mu


def parity(grid):
    """p_l with u_l(beta - tau) = p_l u_l(tau)."""
    return np.sign(grid.u_zero * grid.u_beta)


def energy_ir(grid, G_tau, Sigma_tau):
    """E_dyn = -int_0^beta Tr[G(beta - tau) Sigma(tau)] dtau through the IR coefficients:
    -sum_{l l'} Tr[g_l sigma_l'] int u_l(beta - tau) u_l'(tau) dtau = -sum_l p_l Tr[g_l sigma_l]."""
    n_tau, n, _ = G_tau.shape
    g_l = (grid.fit_tau @ G_tau.reshape(n_tau, n * n)).reshape(-1, n, n)
    s_l = (grid.fit_tau @ Sigma_tau.reshape(n_tau, n * n)).reshape(-1, n, n)
    p = parity(grid)
    return float(-sum(p[l] * np.trace(g_l[l] @ s_l[l]) for l in range(len(p))))


def energy_matsubara(grid, G_tau, Sigma_tau, n_max=20000):
    """E_dyn = (1/beta) sum_n Tr[G(i w_n) Sigma(i w_n)] over |n| <= n_max (Eq. E2b),
    with both functions expanded in the IR basis; the tail beyond n_max is added
    from the leading 1/(i w) moments of the expansions."""
    n_tau, n, _ = G_tau.shape
    beta = grid.basis.beta
    g_l = grid.fit_tau @ G_tau.reshape(n_tau, n * n)
    s_l = grid.fit_tau @ Sigma_tau.reshape(n_tau, n * n)
    nn = np.arange(-n_max - 1, n_max + 1)
    uh = grid.basis.uhat(nn)                       # (L, freqs)
    Gw = (uh.T @ g_l).reshape(-1, n, n)
    Sw = (uh.T @ s_l).reshape(-1, n, n)
    total = np.einsum("wij,wji->", Gw, Sw).real / beta
    # tail: G ~ cG / (i w), Sigma ~ cS / (i w) with c = -(X(0+) + X(beta-)); sum_{|n|>n_max} 1/(i w)^2
    cG = -((grid.u_zero + grid.u_beta) @ g_l).reshape(n, n)
    cS = -((grid.u_zero + grid.u_beta) @ s_l).reshape(n, n)
    w_in = (2 * nn + 1) * np.pi / beta
    tail = -(beta ** 2 / 4.0 - np.sum(1.0 / w_in ** 2))
    return float(total + np.trace(cG @ cS) * tail / beta)


def _diis(history, size):
    """Sum_i c_i out_i with sum_i c_i = 1 minimising |sum_i c_i res_i|^2 (real part of the
    inner products for complex residuals) over the last `size` (out, res) pairs."""
    outs, res = [h[0] for h in history[-size:]], [h[1] for h in history[-size:]]
    k = len(res)
    B = np.empty((k + 1, k + 1))
    B[:k, :k] = [[np.vdot(ri, rj).real for rj in res] for ri in res]
    B[k, :k] = B[:k, k] = -1.0
    B[k, k] = 0.0
    rhs = np.zeros(k + 1)
    rhs[k] = -1.0
    c = np.linalg.lstsq(B, rhs, rcond=None)[0][:k]
    return sum(ci * oi for ci, oi in zip(c, outs))


def run_loop(case, grid, n_elec, tol=1e-8, max_iter=60, damping=0.5, n_damp=2, diis_size=6, mix="diis",
             sigma_fn=None):
    """Self-consistent GF2 loop; returns a dict with the energy history, mu, G, Sigma.

    Monitor energy (F fixed, so the one-body part is 2 Tr[gamma F]):
        E = 2 Tr[gamma F] + E_dyn.
    Mixing: Sigma_in <- damping Sigma_out + (1 - damping) Sigma_in for the first
    n_damp iterations, then DIIS on the residual Sigma_out - Sigma_in
    (mix="damp": damping throughout; mix="cdiis": DIIS on the frequency-dependent
    commutator residual of ``commutator_residual`` instead, extrapolating Sigma_out).
    """
    X, V, F, S = case.X, case.V, case.F, case.S
    n = F.shape[0]
    U = o.thc_U(X, V)
    if sigma_fn is None:
        def sigma_fn(G_tau):
            out = np.empty_like(G_tau)
            for k in range(G_tau.shape[0]):
                Gk = G_tau[k]
                Gm = o.g_minus_tau(G_tau[G_tau.shape[0] - 1 - k])   # mirrored IR grid
                out[k] = o.sigma_sox_thc(X, U, Gk, Gm) + o.sigma_direct_thc(X, V, Gk, Gm)
            return out
    G, mu, Giw = solve_dyson(grid, S, F, None, n_elec, 0.0, return_iw=True)
    Sig_in = np.zeros_like(G)
    hist, E_prev, history = [], None, []
    converged = False
    for it in range(1, max_iter + 1):
        Sig_out = sigma_fn(G)
        E_dyn = energy_ir(grid, G, Sig_out)
        n_tau = G.shape[0]
        g_l = grid.fit_tau @ G.reshape(n_tau, n * n)
        gamma = -(grid.u_beta @ g_l).reshape(n, n)
        E = 2.0 * float(np.trace(gamma @ F)) + E_dyn
        hist.append(dict(iter=it, E=E, E_dyn=E_dyn, mu=mu, n=float(np.trace(gamma @ S))))
        if E_prev is not None and abs(E - E_prev) < tol:
            converged = True
            break
        E_prev = E
        r = commutator_residual(grid, S, F, Giw, Sig_out) if mix == "cdiis" else Sig_out - Sig_in
        history.append((Sig_out, r))
        if mix == "damp" or it <= n_damp:
            Sig_in = damping * Sig_out + (1.0 - damping) * Sig_in
        else:
            Sig_in = _diis(history, diis_size)
        G, mu, Giw = solve_dyson(grid, S, F, Sig_in, n_elec, mu, return_iw=True)
    return dict(history=hist, E=hist[-1]["E"], mu=mu, G=G, Sigma=Sig_out, converged=converged, iters=len(hist))
