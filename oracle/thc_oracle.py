"""Plain FP64 CPU oracle of the THC second-order self-energy.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  It shares no code with the CUDA path; both take their
inputs from the seeded generators in ``workloads``.

Conventions (Sec. II.A of arXiv:2404.17744, read for real orbitals and a
closed-shell restricted reference):

* G_pq(tau) = -<T p(tau) q^dagger>, so for 0 < tau < beta
  G(tau) is negative-definite-like and G(-tau) = -G(beta - tau).
* Chemist-notation integrals from the THC factors (Eq. THC_ERI):
  (pq|rs) = sum_PQ X_pP X_qP V_PQ X_rQ X_sQ, with the paper's core matrix
  U_PQ written V here.
* G and Sigma are per spin; the direct (bubble) term carries the factor -2
  of the closed spin loop, the exchange (SOX) term carries +1.  The paper
  prints the SOX expression (Sec. II.C) with an overall minus sign; with the
  G convention above that sign yields a negative exchange contribution to
  the Galitskii-Migdal energy, opposite to second-order perturbation theory.
  The oracle therefore uses +1, the reading that makes E_dyn[G0] equal twice
  the textbook closed-shell MP2 energy at low temperature; the printed sign
  matches if the paper's "G(-tau)" stands for G(beta - tau).

Two routes are implemented for each term:

* the four-index definitions (feasible for n up to ~10), and
* the paper's THC contraction order for SOX (Sec. II.C, the nine-step
  scheme from U_Pqs to Sigma_tr) and the THC form of the direct term that
  the paper takes over from THC-GW (derived in the docstring of
  ``sigma_direct_thc``).

Pins (tests/test_oracle_pins.py): four-index agreement, one-orbital closed
form, finite-temperature MP2 closed form, zero-temperature textbook MP2,
symmetry, V-scaling, fragment separability; unrestricted: the spin-orbital
four-index definition and the restricted limit; screened term: the weak-coupling
limit, one-orbital closed forms (one spin level, and two different ones
unrestricted), symmetry, the restricted limit of the unrestricted form.
"""
from __future__ import annotations

import numpy as np

# Overall factors of the two second-order terms (per-spin G, restricted).
C_DIRECT = -2.0
C_SOX = +1.0


# ---------------------------------------------------------------- integrals
def eri_from_thc(X: np.ndarray, V: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_PQ X_pP X_qP V_PQ X_rQ X_sQ (Eq. THC_ERI, real factors)."""
    pair = np.einsum("pP,qP->pqP", X, X)
    return np.einsum("pqP,PQ,rsQ->pqrs", pair, V, pair, optimize=True)


def g_minus_tau(G_beta_minus_tau: np.ndarray) -> np.ndarray:
    """G(-tau) = -G(beta - tau) (fermionic antiperiodicity, 0 < tau < beta)."""
    return -G_beta_minus_tau


# ------------------------------------------------ four-index (definition) routes
def sigma_sox_four_index(v: np.ndarray, G: np.ndarray, Gm: np.ndarray) -> np.ndarray:
    """SOX self-energy at one tau from its four-index definition (Sec. II.C).

    Sigma_tr = C_SOX * sum_{pqsuvw} (pr|qs)(tu|vw) G_wp(tau) G_uq(tau) G_sv(-tau)
    G, Gm: n x n arrays G(tau), G(-tau).  Unoptimised einsum: the sum as
    written, one nested loop over all eight indices.
    """
    return C_SOX * np.einsum("prqs,tuvw,wp,uq,sv->tr", v, v, G, G, Gm, optimize=False)


def sigma_direct_four_index(v: np.ndarray, G: np.ndarray, Gm: np.ndarray) -> np.ndarray:
    """Second-order direct (bubble) self-energy at one tau, four-index form.

    Sigma_tr = C_DIRECT * sum (tu|vw)(xr|yz) G_ux(tau) G_vz(tau) G_yw(-tau):
    the interaction line (tu|vw) attaches the external index t, the line
    (xr|yz) the external index r; the bubble closes over (v,w) and (y,z).
    """
    return C_DIRECT * np.einsum("tuvw,xryz,ux,vz,yw->tr", v, v, G, G, Gm, optimize=False)


# ---------------------------------------------------------- THC routes
def thc_U(X: np.ndarray, V: np.ndarray) -> np.ndarray:
    """U_Pqs = sum_Q V_PQ X_qQ X_sQ (Eq. U_contraction), shape N x n x n."""
    N = V.shape[0]
    n = X.shape[0]
    kr = (X[:, None, :] * X[None, :, :]).reshape(n * n, N)  # [(q,s), Q] = X_qQ X_sQ
    return (V @ kr.T).reshape(N, n, n)


def sigma_sox_thc(X: np.ndarray, U: np.ndarray, G: np.ndarray, Gm: np.ndarray,
                  return_intermediates: bool = False):
    """SOX at one tau in the paper's THC order (Sec. II.C scheme).

    Steps, with lower-case AO and upper-case THC indices:
      G_Rq   = sum_u X_uR G_uq(tau)
      G_wP   = sum_p G_wp(tau) X_pP
      A_Pqv  = sum_s U_Pqs G_sv(-tau)
      B_PRv  = sum_q A_Pqv G_Rq
      C_RvP  = sum_w U_Rvw G_wP
      D_PR   = sum_v C_RvP B_PRv
      S_RP   = C_SOX * D_PR
      Sigma_tr = sum_PR X_tR S_RP X_rP
    (The printed summation labels of the two projections are read as sum_u
    and sum_p.)
    """
    G_Rq = X.T @ G
    G_wP = G @ X
    A = np.matmul(U, Gm)                               # [P, q, v]
    B = np.einsum("Pqv,Rq->PRv", A, G_Rq, optimize=True)
    C = np.einsum("Rvw,wP->RvP", U, G_wP, optimize=True)
    D = np.einsum("RvP,PRv->PR", C, B, optimize=True)
    S_RP = C_SOX * D.T
    sigma = X @ S_RP @ X.T
    if return_intermediates:
        return sigma, dict(G_Rq=G_Rq, G_wP=G_wP, A=A, B=B, C=C, D=D)
    return sigma


def sigma_sox_thc_rows(X: np.ndarray, U: np.ndarray, G: np.ndarray, Gm: np.ndarray,
                       rows: int = 64) -> np.ndarray:
    """SOX at one tau by the same steps as ``sigma_sox_thc``, with D_PR formed
    `rows` values of P at a time so that the three-index intermediates B and C
    never exist for all P at once (they are N x N x n each: 25 GB at 500 AOs and
    2500 THC points).  Every step is the formula of the scheme evaluated on a slice
    of P; nothing is reordered or fused.  Pinned to ``sigma_sox_thc`` on small inputs.
    """
    G_Rq = X.T @ G
    G_wP = G @ X
    N = U.shape[0]
    D = np.empty((N, N))
    for p0 in range(0, N, rows):
        sl = slice(p0, min(N, p0 + rows))
        A = np.matmul(U[sl], Gm)                                    # A_Pqv, P in the slice
        B = np.einsum("Pqv,Rq->PRv", A, G_Rq, optimize=True)        # B_PRv
        C = np.einsum("Rvw,wP->RvP", U, G_wP[:, sl], optimize=True)  # C_RvP
        D[sl] = np.einsum("RvP,PRv->PR", C, B, optimize=True)       # D_PR
    S_RP = C_SOX * D.T
    return X @ S_RP @ X.T


def sigma_direct_thc(X: np.ndarray, V: np.ndarray, G: np.ndarray, Gm: np.ndarray) -> np.ndarray:
    """Direct term at one tau in THC form.

    Inserting Eq. THC_ERI into both interaction lines of the direct term,
      Sigma_tr = C_DIRECT * sum_{PQRS} X_tP X_rR V_PQ V_RS G^X_PR(tau) G^X_QS(tau) G^X_SQ(-tau)
    with G^X(tau) = X^T G(tau) X.  Hence, with the polarisation
      Pi_QS = G^X_QS(tau) G^X_SQ(-tau)   and   W = V Pi V,
      Sigma = C_DIRECT * X (G^X(tau) o W) X^T        (o = elementwise).
    """
    GX = X.T @ G @ X
    GXm = X.T @ Gm @ X
    Pi = GX * GXm.T
    W = V @ Pi @ V
    return C_DIRECT * (X @ (GX * W) @ X.T)


def sigma_thc(X: np.ndarray, V: np.ndarray, G_tau: np.ndarray, G_bmt: np.ndarray,
              U: np.ndarray | None = None, terms: str = "both") -> np.ndarray:
    """Sigma(tau_k) = Sigma^dir + Sigma^SOX at every tau point (THC routes).

    G_tau[k] = G(tau_k), G_bmt[k] = G(beta - tau_k); returns n_tau x n x n.
    """
    if U is None and terms in ("both", "sox"):
        U = thc_U(X, V)
    out = np.zeros_like(G_tau)
    for k in range(G_tau.shape[0]):
        G = G_tau[k]
        Gm = g_minus_tau(G_bmt[k])
        if terms in ("both", "sox"):
            out[k] += sigma_sox_thc(X, U, G, Gm)
        if terms in ("both", "direct"):
            out[k] += sigma_direct_thc(X, V, G, Gm)
    return out


def sigma_four_index(v: np.ndarray, G_tau: np.ndarray, G_bmt: np.ndarray, terms: str = "both") -> np.ndarray:
    """Sigma at every tau from the four-index definitions."""
    out = np.zeros_like(G_tau)
    for k in range(G_tau.shape[0]):
        G = G_tau[k]
        Gm = g_minus_tau(G_bmt[k])
        if terms in ("both", "sox"):
            out[k] += sigma_sox_four_index(v, G, Gm)
        if terms in ("both", "direct"):
            out[k] += sigma_direct_four_index(v, G, Gm)
    return out


# ------------------------------------------------------ screened (GW) bubble
def sigma_gw_thc(X: np.ndarray, V: np.ndarray, G_tau: np.ndarray, G_bmt: np.ndarray,
                 to_iw: np.ndarray, to_tau: np.ndarray) -> np.ndarray:
    """Screened direct term of scGW / scGWSOX (Sec. II.C, first paragraph: the THC-GW
    scheme with W screened by the RPA bubble) at every tau point, restricted, per spin.

    With the spin-summed polarisation Pi~(tau) = 2 G^X(tau) o G^X(-tau)^T on the THC
    grid, its bosonic transform Pi~(i Omega), the screened interaction
      W(i Omega) = V [1 - Pi~(i Omega) V]^{-1}
    and its dynamic part W~ = W - V transformed back to tau,
      Sigma^GW(tau) = -X (G^X(tau) o W~(tau)) X^T.
    The first term of W~ = V Pi~ V + V Pi~ V Pi~ V + ... gives the second-order direct
    term of ``sigma_direct_thc``.  to_iw (n_Omega x n_tau) and to_tau (n_tau x n_Omega)
    are the bosonic transforms of the tau grid (workloads.ir.make_bosonic_transforms).
    """
    nt = G_tau.shape[0]
    N = V.shape[0]
    GX = np.stack([X.T @ G_tau[k] @ X for k in range(nt)])
    GXm = np.stack([X.T @ g_minus_tau(G_bmt[k]) @ X for k in range(nt)])
    Pi = 2.0 * GX * np.swapaxes(GXm, 1, 2)
    Pi_iw = np.einsum("mk,kab->mab", to_iw, Pi)
    I = np.eye(N)
    Wt_iw = np.stack([V @ np.linalg.inv(I - P @ V) - V for P in Pi_iw])
    Wt = np.einsum("km,mab->kab", to_tau, Wt_iw)
    return np.stack([-(X @ (GX[k] * Wt[k]) @ X.T) for k in range(nt)])


# ------------------------------------------------- unrestricted (two spins)
def sigma_uhf_spin_orbital(v: np.ndarray, G_a: np.ndarray, G_b: np.ndarray, Gm_a: np.ndarray,
                           Gm_b: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Second-order self-energy of a spin-unrestricted G at one tau, from the
    spin-orbital definition (Sec. II.A works in spin-orbitals).

    The 2n spin-orbitals are (orbital, spin); a chemist-notation integral (pq|rs)
    is the spatial v_pqrs when p, q share a spin and r, s share a spin, else 0;
    G is block-diagonal in spin.  In spin-orbitals the two second-order terms are
      Sigma_tr = - sum (tu|vw)(xr|yz) G_ux G_vz G_yw(-tau)        (bubble)
                 + sum (pr|qs)(tu|vw) G_wp G_uq G_sv(-tau)        (SOX),
    the closed loop of the bubble running over both spins (which gives the -2 of
    the restricted form).  Returns the alpha and beta blocks.  Plain einsum.
    """
    n = v.shape[0]
    spin = np.repeat([0, 1], n)
    orb = np.tile(np.arange(n), 2)
    same = (spin[:, None] == spin[None, :]).astype(float)
    vso = v[np.ix_(orb, orb, orb, orb)] * same[:, :, None, None] * same[None, None, :, :]
    Z = np.zeros_like(G_a)
    G = np.block([[G_a, Z], [Z, G_b]])
    Gm = np.block([[Gm_a, Z], [Z, Gm_b]])
    S = (-np.einsum("tuvw,xryz,ux,vz,yw->tr", vso, vso, G, G, Gm, optimize=False)
         + np.einsum("prqs,tuvw,wp,uq,sv->tr", vso, vso, G, G, Gm, optimize=False))
    return S[:n, :n], S[n:, n:]


def sigma_uhf_thc(X: np.ndarray, V: np.ndarray, U: np.ndarray, G_a: np.ndarray, G_b: np.ndarray,
                  Gm_a: np.ndarray, Gm_b: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Unrestricted self-energies at one tau in THC form.  Per spin s the SOX term is
    the restricted scheme with G^s (all three lines carry spin s); the bubble sums
    the polarisations of both spins and the outer line carries spin s:
      Pi = G^X_a(tau) o G^X_a(-tau)^T + G^X_b(tau) o G^X_b(-tau)^T,
      Sigma^dir_s = -X (G^X_s(tau) o (V Pi V)) X^T."""
    def gx(G):
        return X.T @ G @ X
    Pi = gx(G_a) * gx(Gm_a).T + gx(G_b) * gx(Gm_b).T
    W = V @ Pi @ V
    out = []
    for G, Gm in ((G_a, Gm_a), (G_b, Gm_b)):
        out.append(-(X @ (gx(G) * W) @ X.T) + sigma_sox_thc(X, U, G, Gm))
    return out[0], out[1]


def sigma_gw_uhf_thc(X: np.ndarray, V: np.ndarray, G_tau_a: np.ndarray, G_bmt_a: np.ndarray,
                     G_tau_b: np.ndarray, G_bmt_b: np.ndarray, to_iw: np.ndarray,
                     to_tau: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Screened direct term of an unrestricted G at every tau point (the THC-GW scheme
    of Sec. II.C written for the two spin blocks of the spin-orbital G of Sec. II.A).

    The RPA bubble runs over both spins, each closed loop carrying its own spin:
      Pi~(tau) = G^X_a(tau) o G^X_a(-tau)^T + G^X_b(tau) o G^X_b(-tau)^T,
    one screened interaction W(i Omega) = V [1 - Pi~(i Omega) V]^{-1} serves both
    spins, and the outer line carries spin s:
      Sigma^GW_s(tau) = -X (G^X_s(tau) o W~(tau)) X^T,   W~ = W - V.
    For G_a = G_b this is ``sigma_gw_thc`` for both spins; its first order in the
    bubble is the direct term of ``sigma_uhf_thc``."""
    nt = G_tau_a.shape[0]
    N = V.shape[0]
    GX = [np.stack([X.T @ G[k] @ X for k in range(nt)]) for G in (G_tau_a, G_tau_b)]
    GXm = [np.stack([X.T @ g_minus_tau(Gb[k]) @ X for k in range(nt)]) for Gb in (G_bmt_a, G_bmt_b)]
    Pi = GX[0] * np.swapaxes(GXm[0], 1, 2) + GX[1] * np.swapaxes(GXm[1], 1, 2)
    Pi_iw = np.einsum("mk,kab->mab", to_iw, Pi)
    I = np.eye(N)
    Wt_iw = np.stack([V @ np.linalg.inv(I - P @ V) - V for P in Pi_iw])
    Wt = np.einsum("km,mab->kab", to_tau, Wt_iw)
    a, b = (np.stack([-(X @ (g[k] * Wt[k]) @ X.T) for k in range(nt)]) for g in GX)
    return a, b


def energy_dyn_tau_uhf(G_bmt_a, G_bmt_b, S_a, S_b, weights) -> float:
    """Galitskii-Migdal dynamical energy (Eq. E2b) of an unrestricted G: one half of
    the sum over both spins of -int Tr[G_s(beta - tau) Sigma_s(tau)] dtau (equal to
    the per-spin expression of ``energy_dyn_tau`` when the spins are equal)."""
    return 0.5 * (energy_dyn_tau(G_bmt_a, S_a, weights) + energy_dyn_tau(G_bmt_b, S_b, weights))


# ---------------------------------------------------------------- energy
def energy_dyn_tau(G_bmt: np.ndarray, Sigma_tau: np.ndarray, weights: np.ndarray) -> float:
    """Galitskii-Migdal dynamical energy on the tau axis (Eq. E2b).

    (1/beta) sum_n Tr[G(iw_n) Sigma(iw_n)] = -int_0^beta Tr[G(beta - tau) Sigma(tau)] dtau,
    evaluated with the quadrature weights of the tau grid.  Per spin, as
    written in Eq. E2b for the restricted G: the spin sum and the 1/2 of the
    Galitskii-Migdal formula cancel.
    """
    tr = np.array([np.trace(G_bmt[k] @ Sigma_tau[k]) for k in range(G_bmt.shape[0])])
    return float(-np.dot(weights, tr))


# ----------------------------------------------------- noninteracting G
def fermi_pair(e: np.ndarray, beta: float) -> tuple[np.ndarray, np.ndarray]:
    """(n, 1 - n) for occupation n = 1/(1 + e^{beta e}), both computed without cancellation."""
    t = np.tanh(0.5 * beta * e)
    return 0.5 * (1.0 - t), 0.5 * (1.0 + t)


def g0_tau(F: np.ndarray, S: np.ndarray, mu: float, beta: float, tau: np.ndarray) -> np.ndarray:
    """Noninteracting G(tau) from Dyson with Sigma = 0 (Sec. II.A).

    G(iw) = [(iw + mu) S - F]^{-1}; with F C = S C diag(eps), C^T S C = I,
    G(tau) = -C diag((1 - n_k) e^{-e'_k tau}) C^T, e' = eps - mu.  The factor
    is written as exp(-e' tau) (1-n) for e' >= 0 and exp(e'(beta - tau)) n
    for e' < 0, the two equal forms that never overflow.
    """
    import scipy.linalg

    eps, C = scipy.linalg.eigh(F, S)
    e = eps - mu
    n_occ, n_vir = fermi_pair(e, beta)
    out = np.empty((len(tau), F.shape[0], F.shape[0]))
    pos = e >= 0.0
    for k, t in enumerate(tau):
        f = np.empty_like(e)
        f[pos] = np.exp(-e[pos] * t) * n_vir[pos]
        f[~pos] = np.exp(e[~pos] * (beta - t)) * n_occ[~pos]
        out[k] = -(C * f[None, :]) @ C.T
    return out


# -------------------------------------------------------- closed forms
def one_orbital_sigma(v: float, e: float, beta: float, tau: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(Sigma^dir, Sigma^SOX) for a single orbital with (00|00) = v, e = eps - mu.

    With G(tau) = -(1-n) e^{-e tau}, G(-tau) = n e^{e tau}, both terms are
    v^2 G(tau)^2 G(-tau) times their factor: (1-n)^2 n e^{-e tau} v^2 times
    C_DIRECT and C_SOX.
    """
    n_occ, n_vir = fermi_pair(np.array([e]), beta)
    base = v * v * n_vir[0] ** 2 * n_occ[0] * np.exp(-e * tau)
    return C_DIRECT * base, C_SOX * base


def _pair_weight(e_in1, e_in2, e_out1, e_out2, beta):
    """w = [n_in1 n_in2 nbar_out1 nbar_out2 - nbar_in1 nbar_in2 n_out1 n_out2] / Delta,
    Delta = e_out1 + e_out2 - e_in1 - e_in2, with the Delta -> 0 limit
    beta n_in1 n_in2 nbar_out1 nbar_out2.  Arguments broadcast."""
    n1, nb1 = fermi_pair(e_in1, beta)
    n2, nb2 = fermi_pair(e_in2, beta)
    n3, nb3 = fermi_pair(e_out1, beta)
    n4, nb4 = fermi_pair(e_out2, beta)
    a = n1 * n2 * nb3 * nb4
    b = nb1 * nb2 * n3 * n4
    delta = e_out1 + e_out2 - e_in1 - e_in2
    small = np.abs(delta) < 1e-12
    safe = np.where(small, 1.0, delta)
    return np.where(small, beta * a, (a - b) / safe)


def mp2_finite_T(v_mo: np.ndarray, e: np.ndarray, beta: float) -> tuple[float, float]:
    """(E^dir_dyn, E^SOX_dyn) of the GM energy at G0, closed form in the eigenbasis.

    Derivation: with diagonal G0, -int_0^beta Tr[G(beta - tau) Sigma(tau)] reduces
    to single exponentials in tau, integrated analytically:
      E^dir = C_DIRECT * sum_{tuvw} (tu|vw)^2 w(t, w -> u, v)
      E^SOX = C_SOX    * sum_{ptqv} (pt|qv)(tq|vp) w(t, v -> p, q)
    where w(a, b -> c, d) is ``_pair_weight`` with Delta = e_c + e_d - e_a - e_b.
    v_mo are the integrals in the orthonormal eigenbasis, e = eps - mu.
    """
    et = e[:, None, None, None]
    eu = e[None, :, None, None]
    ev = e[None, None, :, None]
    ew = e[None, None, None, :]
    # direct: indices (t,u,v,w), in = (t, w), out = (u, v)
    w_dir = _pair_weight(et, ew, eu, ev, beta)
    E_dir = C_DIRECT * float(np.sum(v_mo ** 2 * w_dir))
    # exchange: indices (p,t,q,v) of (pt|qv); in = (t, v), out = (p, q)
    ep = e[:, None, None, None]
    et2 = e[None, :, None, None]
    eq = e[None, None, :, None]
    ev2 = e[None, None, None, :]
    w_x = _pair_weight(et2, ev2, ep, eq, beta)
    prod = v_mo * np.einsum("tqvp->ptqv", v_mo)  # (pt|qv) * (tq|vp)
    E_x = C_SOX * float(np.sum(prod * w_x))
    return E_dir, E_x


def mp2_zero_T_closed_shell(v_mo: np.ndarray, eps: np.ndarray, n_occ: int) -> float:
    """Textbook closed-shell MP2 energy
    sum_{ijab} (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b)."""
    o = slice(0, n_occ)
    vv = slice(n_occ, len(eps))
    iajb = v_mo[o, vv, o, vv]
    eo = eps[o]
    ev = eps[vv]
    denom = eo[:, None, None, None] + eo[None, None, :, None] - ev[None, :, None, None] - ev[None, None, None, :]
    ibja = np.einsum("ibja->iajb", v_mo[o, vv, o, vv])
    return float(np.sum(iajb * (2.0 * iajb - ibja) / denom))


def mo_eri(v: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Integrals in the basis of the columns of C: (ab|cd) = sum C_pa C_qb C_rc C_sd (pq|rs)."""
    return np.einsum("pqrs,pa,qb,rc,sd->abcd", v, C, C, C, C, optimize=True)


# ---------------------------------------------------------- tau quadrature
def composite_gauss_legendre(beta: float, n_panels_per_side: int = 24, order: int = 24,
                             smallest: float = 1e-6) -> tuple[np.ndarray, np.ndarray]:
    """Mirror-symmetric composite Gauss-Legendre rule on (0, beta).

    Panels are geometrically graded towards both ends, where G(tau) and
    Sigma(tau) vary as e^{-|e| tau} on scales down to 1/|e|.
    """
    half = 0.5 * beta
    edges = np.concatenate([[0.0], half * np.geomspace(smallest / half, 1.0, n_panels_per_side)])
    x, w = np.polynomial.legendre.leggauss(order)
    nodes = []
    weights = []
    for a, b in zip(edges[:-1], edges[1:]):
        nodes.append(0.5 * (b - a) * x + 0.5 * (a + b))
        weights.append(0.5 * (b - a) * w)
    left = np.concatenate(nodes)
    wl = np.concatenate(weights)
    tau = np.concatenate([left, beta - left[::-1]])
    wts = np.concatenate([wl, wl[::-1]])
    return tau, wts
