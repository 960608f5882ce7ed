"""Seeded synthetic inputs for the THC self-energy workloads.

This module only draws inputs: random THC factors X and V, a Fock matrix F,
an overlap S, a mirror-symmetric imaginary-time grid and the noninteracting
Green's function of (F, S, mu) on that grid.  It holds none of the
self-energy arithmetic, so the CUDA path and the CPU oracle can both take
their inputs from here without sharing any of the method.

Recipe (stands in for the paper's S22 / aug-cc-pVTZ molecules, whose
integrals and geometries are not available; Sec. III.A gives beta = 1000,
Sec. III.B gives alpha = N/n between 5 and 10):

* X_iP ~ Normal(mean 0, standard deviation n^{-1/2}), shape n x N
  (collocation matrix of the THC factorisation, Eq. THC_ERI).
* V = Q diag(10^u) Q^T, u ~ Uniform[-3, 0], Q Haar-orthogonal: symmetric
  positive definite like the LS-THC core V = A^T A (Sec. II.B).
* F = S^{1/2} Q diag(eps) Q^T S^{1/2} with eps drawn per workload, so that
  the generalised eigenvalues of (F, S) are exactly eps.
* S = I, or I + 0.1 M / ||M||_2 with M random SPD.
* tau grid: Gauss-Legendre nodes on (0, beta) (mirror-symmetric, so
  G(beta - tau_k) is G at node n_tau - 1 - k).
* G(tau) = -C diag(e^{-e' tau} / (1 + e^{-beta e'})) C^T with C^T S C = I,
  e' = eps - mu; written in branch-stable form.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 17744


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 generator for a workload seed."""
    return np.random.Generator(np.random.PCG64(seed))


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian, signs fixed)."""
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    q = q * np.sign(np.diag(r))[None, :]
    return q


def draw_X(n: int, N: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal((n, N)) / np.sqrt(n)


def draw_V(N: int, rng: np.random.Generator, log10_lo: float = -3.0, log10_hi: float = 0.0) -> np.ndarray:
    q = haar_orthogonal(N, rng)
    lam = 10.0 ** rng.uniform(log10_lo, log10_hi, size=N)
    V = (q * lam[None, :]) @ q.T
    return 0.5 * (V + V.T)


def draw_S(n: int, rng: np.random.Generator, identity: bool) -> np.ndarray:
    if identity:
        return np.eye(n)
    m = rng.standard_normal((n, n))
    m = m @ m.T
    S = np.eye(n) + 0.1 * m / np.linalg.norm(m, 2)
    return 0.5 * (S + S.T)


def sym_sqrt(S: np.ndarray) -> np.ndarray:
    w, q = np.linalg.eigh(S)
    return (q * np.sqrt(w)[None, :]) @ q.T


def draw_F(eps: np.ndarray, S: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    n = eps.shape[0]
    q = haar_orthogonal(n, rng)
    h = sym_sqrt(S)
    F = h @ ((q * eps[None, :]) @ q.T) @ h
    return 0.5 * (F + F.T)


def gauss_legendre_tau(n_tau: int, beta: float) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre nodes and weights mapped to (0, beta), ascending."""
    x, w = np.polynomial.legendre.leggauss(n_tau)
    tau = 0.5 * beta * (x + 1.0)
    tau = 0.5 * (tau + (beta - tau[::-1]))  # exact mirror symmetry in floating point
    return tau, 0.5 * beta * w


def noninteracting_G(F: np.ndarray, S: np.ndarray, mu: float, beta: float, tau: np.ndarray) -> np.ndarray:
    """G(tau) of the independent-particle Hamiltonian (F, S) at chemical potential mu.

    Returns an array of shape (len(tau), n, n); every tau must lie in [0, beta].
    """
    h_inv = np.linalg.inv(sym_sqrt(S))
    w, q = np.linalg.eigh(h_inv @ F @ h_inv)
    C = h_inv @ q  # C^T S C = I, F C = S C diag(w)
    e = w - mu
    out = np.empty((len(tau), F.shape[0], F.shape[0]))
    pos = e >= 0.0
    denom = 1.0 + np.exp(-beta * np.abs(e))
    for k, t in enumerate(tau):
        f = np.empty_like(e)
        f[pos] = np.exp(-e[pos] * t) / denom[pos]
        f[~pos] = np.exp(e[~pos] * (beta - t)) / denom[~pos]
        out[k] = -(C * f[None, :]) @ C.T
    return out


@dataclasses.dataclass
class SigmaCase:
    """One single-evaluation workload: inputs of the self-energy."""
    n: int
    N: int
    n_tau: int
    beta: float
    mu: float
    X: np.ndarray          # n x N
    V: np.ndarray          # N x N
    F: np.ndarray          # n x n
    S: np.ndarray          # n x n
    eps: np.ndarray        # generalised eigenvalues of (F, S)
    tau: np.ndarray        # n_tau, ascending, mirror-symmetric
    tau_w: np.ndarray      # quadrature weights on (0, beta)
    G_tau: np.ndarray      # n_tau x n x n
    G_bmt: np.ndarray      # G(beta - tau_k), n_tau x n x n

    def mirror_index(self) -> np.ndarray:
        return np.arange(self.n_tau)[::-1].copy()


def make_sigma_case(n: int, N: int, n_tau: int, beta: float, seed: int,
                    identity_S: bool = True, n_occ: int | None = None,
                    eps_range: tuple[float, float] = (-2.0, 2.0),
                    mu: float = 0.0) -> SigmaCase:
    """Seeded single-evaluation workload.

    With n_occ None the orbital energies are Uniform[eps_range]; otherwise
    n_occ of them are Uniform[-2, -0.1] and the rest Uniform[0.1, 2] (a gap
    around mu = 0, the recipe of the 200-AO loop workload).
    """
    rng = rng_for(seed)
    if n_occ is None:
        eps = np.sort(rng.uniform(eps_range[0], eps_range[1], size=n))
    else:
        eps = np.sort(np.concatenate([rng.uniform(-2.0, -0.1, size=n_occ),
                                      rng.uniform(0.1, 2.0, size=n - n_occ)]))
    S = draw_S(n, rng, identity_S)
    F = draw_F(eps, S, rng)
    X = draw_X(n, N, rng)
    V = draw_V(N, rng)
    tau, tau_w = gauss_legendre_tau(n_tau, beta)
    G_tau = noninteracting_G(F, S, mu, beta, tau)
    G_bmt = G_tau[::-1].copy()
    return SigmaCase(n, N, n_tau, beta, mu, X, V, F, S, eps, tau, tau_w, G_tau, G_bmt)


# Named workloads (n, N, n_tau, beta) of the benchmark table.
WORKLOADS = {
    "thc20":   dict(n=20,   N=60,   n_tau=32,  beta=100.0,  seed=SEED_BASE + 1),
    "thc200":  dict(n=200,  N=1000, n_tau=100, beta=100.0,  seed=SEED_BASE + 2, identity_S=False, n_occ=40),
    # the same system on 4 tau points: small profiling case (U_Pqs = 320 MB still exceeds L2)
    "thc200s": dict(n=200,  N=1000, n_tau=4,   beta=100.0,  seed=SEED_BASE + 2, identity_S=False, n_occ=40),
    "thc500":  dict(n=500,  N=2500, n_tau=120, beta=1000.0, seed=SEED_BASE + 3),
    "thc1100": dict(n=1100, N=5500, n_tau=100, beta=1000.0, seed=SEED_BASE + 5),
}


def make_workload(name: str, **override) -> SigmaCase:
    kw = dict(WORKLOADS[name])
    kw.update(override)
    return make_sigma_case(**kw)


def random_symmetric(n_tau: int, n: int, rng: np.random.Generator, scale: float = 1.0) -> np.ndarray:
    """Random symmetric matrices (for tests that need generic, non-physical G)."""
    a = rng.standard_normal((n_tau, n, n)) * scale
    return 0.5 * (a + np.swapaxes(a, 1, 2))
