"""Intermediate-representation (IR) basis and sparse sampling grids, from scratch.

The paper runs its self-consistency on the IR basis with sparse sampling
(Sec. III.A: beta = 1000, Lambda = 1e5, via sparse-ir).  sparse-ir is not
available here, so this module constructs the fermionic IR basis from its
published definition (Shinaoka et al., PRB 96, 035147 (2017); Li et al., PRB
101, 035144 (2020)):

* the logistic kernel K(tau, w) = e^{-tau w} / (1 + e^{-beta w}) on
  tau in [0, beta], w in [-w_max, w_max] is discretised with composite
  Gauss-Legendre rules on geometrically graded panels (tau: towards 0 and beta;
  w: towards 0 and +-w_max), so that Lambda = beta w_max up to 1e5 (Sec. III.A)
  builds in seconds;
* the SVD of the quadrature-weighted kernel gives the singular values s_l
  and the basis functions u_l(tau), orthonormal on [0, beta], kept while
  s_l / s_0 >= eps;
* u_l is a degree-(order - 1) polynomial on every tau panel (its values at
  the panel's Gauss nodes), so u_l(tau) anywhere is the panel's Legendre
  interpolant and its Fourier transform uhat_l(i w_n) = int e^{i w_n tau}
  u_l(tau) dtau is exact per panel through spherical Bessel functions;
* tau sampling points: the L roots of u_L; Matsubara sampling points: the
  sign changes of uhat_{L-1}(i w_n) over n >= 0, mirrored to n < 0.

Like the tau grid, the basis and its sampling matrices are inputs of the
self-energy loop: both the CUDA loop and the oracle loop take them from here
and do their own arithmetic with them.  This module holds no self-energy
arithmetic.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.special


def _graded_panels(a: float, b: float, smallest: float, per_decade: int, center: bool) -> np.ndarray:
    """Panel edges on [a, b], geometric with per_decade panels per decade from `smallest`,
    towards both ends (the tau interval: the basis functions vary on 1/w_max next to 0
    and beta) and, with center, also towards the midpoint (the w interval: the kernel
    switches on the scale 1/beta around w = 0)."""
    half = 0.5 * (b - a)
    if not center:
        nd = max(1, int(np.ceil(per_decade * np.log10(half / smallest))))
        g = np.concatenate([[0.0], np.geomspace(smallest, half, nd + 1)])
        return np.unique(np.concatenate([a + g, b - g]))
    m, q = 0.5 * (a + b), 0.5 * half
    nd = max(1, int(np.ceil(per_decade * np.log10(q / smallest))))
    g = np.concatenate([[0.0], np.geomspace(smallest, q, nd + 1)])
    return np.unique(np.concatenate([m + g, b - g, m - g, a + g]))


def _gauss_on_panels(edges: np.ndarray, order: int):
    x, w = np.polynomial.legendre.leggauss(order)
    nodes, weights = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        nodes.append(0.5 * (b - a) * x + 0.5 * (a + b))
        weights.append(0.5 * (b - a) * w)
    return np.concatenate(nodes), np.concatenate(weights)


def logistic_kernel(tau: np.ndarray, w: np.ndarray, beta: float) -> np.ndarray:
    """K(tau, w) = e^{-tau w} / (1 + e^{-beta w}) without overflow."""
    t = tau[:, None]
    ww = w[None, :]
    pos = ww >= 0
    out = np.empty((len(tau), len(w)))
    ep = np.exp(-t * np.where(pos, ww, 0.0)) / (1.0 + np.exp(-beta * np.where(pos, ww, 0.0)))
    en = np.exp((beta - t) * np.where(pos, 0.0, ww)) / (1.0 + np.exp(beta * np.where(pos, 0.0, ww)))
    out[:] = np.where(pos, ep, en)
    return out


@dataclasses.dataclass
class IRBasis:
    beta: float
    wmax: float
    eps: float
    s: np.ndarray            # singular values, length L
    edges: np.ndarray        # tau panel edges
    order: int               # Gauss points per panel
    coef: np.ndarray         # Legendre coefficients per panel: (L, n_panels, order)
    tau_s: np.ndarray        # tau sampling points (L)
    n_s: np.ndarray          # Matsubara sampling indices n (w_n = (2n+1) pi / beta)

    @property
    def L(self) -> int:
        return len(self.s)

    @property
    def iw_s(self) -> np.ndarray:
        return (2 * self.n_s + 1) * np.pi / self.beta

    # ------------------------------------------------------- evaluation
    def u(self, tau: np.ndarray) -> np.ndarray:
        """u_l(tau), shape (L, len(tau)); tau in [0, beta]."""
        tau = np.atleast_1d(np.asarray(tau, dtype=float))
        p = np.clip(np.searchsorted(self.edges, tau, side="right") - 1, 0, len(self.edges) - 2)
        a, b = self.edges[p], self.edges[p + 1]
        x = np.clip((2 * tau - a - b) / (b - a), -1.0, 1.0)
        P = np.polynomial.legendre.legvander(x, self.order - 1)  # (len(tau), order)
        return np.einsum("lto,to->lt", self.coef[:, p, :], P)

    def uhat(self, n: np.ndarray) -> np.ndarray:
        """uhat_l(i w_n) = int_0^beta e^{i w_n tau} u_l(tau) dtau, shape (L, len(n)), exact per panel."""
        n = np.atleast_1d(np.asarray(n))
        return self.uhat_w((2 * n + 1) * np.pi / self.beta)

    def uhat_w(self, w: np.ndarray) -> np.ndarray:
        """int_0^beta e^{i w tau} u_l(tau) dtau at real frequencies w, shape (L, len(w))."""
        w = np.atleast_1d(np.asarray(w, dtype=float))
        a, b = self.edges[:-1], self.edges[1:]
        c, h = 0.5 * (a + b), 0.5 * (b - a)
        # int_a^b e^{i w tau} P_p(x(tau)) dtau = 2 h e^{i w c} i^p j_p(w h)
        z = w[None, :] * h[:, None]                          # (panels, freqs)
        phase = np.exp(1j * w[None, :] * c[:, None]) * 2 * h[:, None]
        out = np.zeros((self.L, len(w)), dtype=complex)
        for p in range(self.order):
            jp = scipy.special.spherical_jn(p, z) * (1j ** p)  # (panels, freqs)
            out += self.coef[:, :, p] @ (phase * jp)
        return out


def build_ir(beta: float, wmax: float, eps: float = 1e-10, order: int = 16, L_max: int | None = None) -> IRBasis:
    """Constructs the fermionic IR basis for (beta, wmax) and its sampling grids."""
    lam = beta * wmax
    t_edges = _graded_panels(0.0, beta, smallest=min(0.05 / wmax, beta / 1e3), per_decade=4, center=False)
    w_edges = _graded_panels(-wmax, wmax, smallest=min(0.05 / beta, wmax / 1e3), per_decade=4, center=True)
    tn, tw = _gauss_on_panels(t_edges, order)
    wn, ww = _gauss_on_panels(w_edges, order)
    A = np.sqrt(tw)[:, None] * logistic_kernel(tn, wn, beta) * np.sqrt(ww)[None, :]
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    keep = s / s[0] >= eps
    L = int(np.sum(keep))
    if L_max is not None:
        L = min(L, L_max)
    # values of u_l at the tau nodes (orthonormal in L2[0, beta]); one extra for the sampling roots
    Lx = L + 1
    uval = U[:, :Lx] / np.sqrt(tw)[:, None]
    # sign convention: u_l(beta) > 0
    uval *= np.sign(uval[-1, :])[None, :]
    n_pan = len(t_edges) - 1
    x, _ = np.polynomial.legendre.leggauss(order)
    Vinv = np.linalg.inv(np.polynomial.legendre.legvander(x, order - 1))
    # Legendre coefficients of u_l on every panel: (Lx, panels, order)
    coef_all = np.einsum("po,lko->lkp", Vinv, uval.T.reshape(Lx, n_pan, order))
    basis_x = IRBasis(beta, wmax, eps, s[:Lx], t_edges, order, coef_all, np.empty(0), np.empty(0, dtype=int))
    # tau sampling: roots of u_L (parity makes them mirror-symmetric)
    grid = np.linspace(0.0, beta, 200 * Lx + 1)
    grid = np.unique(np.concatenate([grid, tn]))
    uL = basis_x.u(grid)[L]
    roots = []
    for i in np.nonzero(np.sign(uL[:-1]) * np.sign(uL[1:]) < 0)[0]:
        lo, hi = grid[i], grid[i + 1]
        flo = uL[i]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            fm = basis_x.u(np.array([mid]))[L, 0]
            if np.sign(fm) == np.sign(flo):
                lo, flo = mid, fm
            else:
                hi = mid
        roots.append(0.5 * (lo + hi))
    tau_s = np.array(sorted(roots))
    tau_s = 0.5 * (tau_s + (beta - tau_s[::-1]))  # exact mirror symmetry
    # Matsubara sampling: sign changes of uhat_{L-1} over n >= 0 (real or imaginary by parity)
    n_max = int(max(4 * L, 2 * lam / np.pi + 10 * L))
    nn = np.arange(0, n_max)
    uh = basis_x.uhat(nn)[L - 1]
    f = uh.real if np.abs(uh.real).max() > np.abs(uh.imag).max() else uh.imag
    ch = np.nonzero(np.sign(f[:-1]) * np.sign(f[1:]) < 0)[0]
    pos = sorted(set([0] + [int(i) + 1 for i in ch] + [n_max - 1]))
    n_s = np.array(sorted(set([-p - 1 for p in pos] + pos)))
    return IRBasis(beta, wmax, eps, s[:L], t_edges, order, coef_all[:L], tau_s, n_s)


@dataclasses.dataclass
class LoopGrid:
    """Matrices of the sparse-sampling transforms used by the self-consistency loop."""
    basis: IRBasis
    tau: np.ndarray          # n_tau sampling points
    n: np.ndarray            # Matsubara indices
    iw: np.ndarray           # w_n
    U_tau: np.ndarray        # (n_tau, L): G(tau_k) = sum_l U_tau[k, l] g_l
    fit_tau: np.ndarray      # (L, n_tau): g_l = sum_k fit_tau[l, k] G(tau_k)
    U_iw: np.ndarray         # (n_iw, L) complex: G(i w_m) = sum_l U_iw[m, l] g_l
    fit_iw: np.ndarray       # (L, n_iw) complex: g_l = sum_m fit_iw[l, m] G(i w_m)
    u_beta: np.ndarray       # (L,) u_l(beta^-), so G(beta^-) = sum_l u_beta[l] g_l
    u_zero: np.ndarray       # (L,) u_l(0^+)


def make_loop_grid(beta: float, wmax: float, eps: float = 1e-10, L_max: int | None = None) -> LoopGrid:
    b = build_ir(beta, wmax, eps=eps, L_max=L_max)
    U_tau = b.u(b.tau_s).T
    U_iw = b.uhat(b.n_s).T
    fit_tau = np.linalg.pinv(U_tau)
    fit_iw = np.linalg.pinv(U_iw)
    ub = b.u(np.array([beta]))[:, 0]
    u0 = b.u(np.array([0.0]))[:, 0]
    return LoopGrid(b, b.tau_s, b.n_s, b.iw_s, U_tau, fit_tau, U_iw, fit_iw, ub, u0)


@dataclasses.dataclass
class BosonicTransforms:
    """Bosonic Matsubara transforms of functions sampled on a loop grid's tau points.

    The screened interaction of GW (Sec. II.C names scGW and scGWSOX) needs the
    polarisation Pi(tau) at bosonic frequencies i Omega_m = 2 pi m i / beta and the
    screened W(i Omega) back on the tau grid.  Pi(tau) and W(tau) of real symmetric
    matrices are real, symmetric under tau -> beta - tau, and their transforms are
    real and even in Omega, so they are expanded in the even-parity functions u_l of
    the grid's basis (which span e^{-w tau} + e^{-w (beta - tau)} for |w| <= w_max as
    well as the odd-parity ones span the antisymmetric part), and sampled at m >= 0:
      f(i Omega_m) = sum_k to_iw[m, k] f(tau_k),    f(tau_k) = sum_m to_tau[k, m] f(i Omega_m).
    """
    m: np.ndarray            # bosonic Matsubara indices (>= 0)
    omega: np.ndarray        # Omega_m = 2 pi m / beta
    to_iw: np.ndarray        # (n_Omega, n_tau) real
    to_tau: np.ndarray       # (n_tau, n_Omega) real


def make_bosonic_transforms(grid: LoopGrid) -> BosonicTransforms:
    """Sampling matrices of the bosonic transforms on grid.tau.

    R[m, l] = Re int_0^beta e^{i Omega_m tau} u_l(tau) dtau for the even-parity u_l;
    the sampled m are 0, the sign changes of R[., l_e] of the highest even function
    l_e over m < m_max, and m_max - 1 (the construction of the fermionic sampling,
    applied to the even cosine transform), extended by the midpoints of the widest
    gaps until there are at least as many frequencies as even functions."""
    b = grid.basis
    even = np.nonzero(grid.u_zero * grid.u_beta > 0)[0]
    beta = b.beta
    m_max = int(max(4 * b.L, b.beta * b.wmax / np.pi + 10 * b.L))
    mm = np.arange(0, m_max)
    R_all = b.uhat_w(2 * np.pi * mm / beta)[even].real        # (L_e, m_max)
    f = R_all[-1]
    ch = np.nonzero(np.sign(f[:-1]) * np.sign(f[1:]) < 0)[0]
    sel = sorted(set([0] + [int(i) + 1 for i in ch] + [m_max - 1]))
    while len(sel) < len(even):
        gaps = np.diff(sel)
        i = int(np.argmax(gaps))
        sel.insert(i + 1, (sel[i] + sel[i + 1]) // 2)
        sel = sorted(set(sel))
    m = np.array(sel)
    R = R_all[:, m].T                                          # (n_Omega, L_e)
    to_iw = R @ grid.fit_tau[even, :]
    to_tau = grid.U_tau[:, even] @ np.linalg.pinv(R)
    return BosonicTransforms(m, 2 * np.pi * m / beta, to_iw, to_tau)
