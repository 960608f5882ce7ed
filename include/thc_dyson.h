/*
 * thc_dyson.h -- C ABI of the Dyson step of the GPU self-consistency loop.
 *
 * One iteration of fully self-consistent GF2 (Sec. II.A of arXiv:2404.17744)
 * evaluates Sigma(tau) (thc_sigma.h), then solves the Dyson equation in the
 * non-orthogonal AO basis (Eq. Dyson),
 *     G(i w_n) = [(i w_n + mu) S - F - Sigma(i w_n)]^{-1},
 * with mu re-optimised so that the electron count is fixed (appendix, case 2),
 * and transforms G back to the tau grid.  The tau <-> i w transforms are
 * sparse-sampling matrices of an intermediate-representation (IR) basis
 * (Sec. III.A) supplied by the caller:
 *     g_l = sum_k fit_tau[l][k] X(tau_k),   X(tau_k) = sum_l U_tau[k][l] g_l,
 *     X(i w_m) = sum_l U_iw[m][l] g_l,      g_l = sum_m fit_iw[l][m] X(i w_m).
 * F is the fixed one-body (Fock) matrix; Sigma is the dynamical part only.
 * Everything runs in FP64 on the GPU; all matrices are row-major.  Return
 * codes are those of thc_sigma.h; failures are described by
 * thc_dyson_last_error(d) (or thc_last_error(NULL) when d is NULL).
 */
#ifndef THC_DYSON_H
#define THC_DYSON_H

#include "thc_sigma.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thc_dyson thc_dyson;   /* opaque, library-owned */

/*
 * thc_dyson_init -- set up the Dyson step.
 *   n_ao, n_tau, n_iw, n_l  sizes (n_l basis functions; n_ao <= 1500)
 *   beta          inverse temperature
 *   S, F          host or dev, n_ao x n_ao overlap and one-body matrices (copied)
 *   U_tau         host, n_tau x n_l;  fit_tau host, n_l x n_tau
 *   U_iw          host, n_iw x n_l complex, interleaved (re, im)
 *   fit_iw        host, n_l x n_iw complex, interleaved (re, im)
 *   iw            host, n_iw fermionic Matsubara frequencies w_m
 *   u_beta, u_zero host, n_l values u_l(beta^-) and u_l(0^+) of the basis
 *   stream        cudaStream_t (NULL: legacy default stream)
 */
int thc_dyson_init(thc_dyson **d, int n_ao, int n_tau, int n_iw, int n_l, double beta,
                   const double *S, const double *F, const double *U_tau, const double *fit_tau,
                   const double *U_iw, const double *fit_iw, const double *iw,
                   const double *u_beta, const double *u_zero, void *stream);

/*
 * thc_dyson_solve -- G(tau) from Sigma(tau) at fixed electron count.
 *   Sigma_tau  dev, n_tau x n_ao x n_ao (NULL: Sigma = 0, the noninteracting G)
 *   n_elec     target electron count per spin, Tr[gamma S] with gamma = -G(beta^-)
 *   mu         in: starting guess; out: the chemical potential found
 *   tol        tolerance on the electron count (<= 0: 1e-10)
 *   G_tau      dev out, n_tau x n_ao x n_ao
 * The count N(mu) is monotonic; the search takes Newton steps on the analytic
 * slope dN/dmu (see thc_dyson_count), capped at 0.5 Ha, kept inside a bracket
 * once one is known and safeguarded by bisection (each trial is a full set of
 * n_iw complex inversions).  THC_EINVAL if it does not converge.  Synchronises.
 */
int thc_dyson_solve(thc_dyson *d, const double *Sigma_tau, double n_elec, double *mu, double tol,
                    double *G_tau);

/*
 * thc_dyson_energy -- energies from tau-grid data through the IR coefficients:
 *   E_dyn = -int_0^beta Tr[G(beta - tau) Sigma(tau)] dtau = -sum_l p_l Tr[g_l sigma_l]
 * (Eq. E2b per spin; p_l = +-1 the parity u_l(beta - tau) = p_l u_l(tau)),
 *   gamma_F = Tr[gamma F] and n_per_spin = Tr[gamma S], gamma = -G(beta^-).
 * G_tau, Sigma_tau dev; outputs host (gamma_F, n_per_spin may be NULL).  Synchronises.
 */
int thc_dyson_energy(thc_dyson *d, const double *G_tau, const double *Sigma_tau, double *E_dyn,
                     double *gamma_F, double *n_per_spin);

/*
 * thc_dyson_count -- electron count per spin N(mu) = Tr[gamma S] of the Green's
 * function G(i w) = [(i w + mu) S - F - Sigma(i w)]^{-1} at the given mu (appendix,
 * case 2), and its slope dN/dmu = -Tr[(d gamma / dmu) S] from dG/dmu = -G S G
 * (the slope thc_dyson_solve's Newton steps use).
 *   Sigma_tau  dev, n_tau x n_ao x n_ao (NULL: Sigma = 0)
 *   mu         chemical potential
 *   n_per_spin host out;  dn_dmu host out (may be NULL)
 * Overwrites the G(i w) that thc_dyson_commutator reads.  Synchronises.
 */
int thc_dyson_count(thc_dyson *d, const double *Sigma_tau, double mu, double *n_per_spin,
                    double *dn_dmu);

/*
 * thc_dyson_commutator -- frequency-dependent commutator residual of the
 * self-consistency, the error vector of commutator DIIS (Sec. III.A names damping
 * and a frequency-dependent commutator DIIS):
 *   e(i w_m) = H_m G_m S - S G_m H_m,   H_m = F + Sigma_out(i w_m),
 * for every sampled frequency, with G_m the G(i w_m) of the last thc_dyson_solve
 * (the Green's function Sigma_out was evaluated from).  At self-consistency
 * G^{-1} = (i w + mu) S - H, so e = 0.
 *   Sigma_out_tau dev, n_tau x n_ao x n_ao
 *   E_iw          dev out, n_iw x n_ao x n_ao complex, interleaved (re, im)
 * Allocates an n_iw x n_ao^2 complex workspace on first use (kept by d).
 * Stream-ordered.
 */
int thc_dyson_commutator(thc_dyson *d, const double *Sigma_out_tau, double *E_iw);

/* thc_dyson_evals -- number of N(mu) evaluations in the last thc_dyson_solve. */
int thc_dyson_evals(const thc_dyson *d);

/* thc_dyson_last_error -- text of the last failure on d ("" when none). */
const char *thc_dyson_last_error(const thc_dyson *d);

/* thc_dyson_destroy -- free d (NULL is a no-op).  Synchronises. */
void thc_dyson_destroy(thc_dyson *d);

/*
 * thc_vec_dot -- *out = sum_i x[i] y[i] over len FP64 device values, in a
 * fixed reduction order (deterministic).  scratch: dev, >= 257 doubles.
 * Synchronises the stream.  (Mixing and DIIS of the loop; no paper counterpart.)
 */
int thc_vec_dot(long long len, const double *x, const double *y, double *scratch, double *out,
                void *stream);

/*
 * thc_vec_lincomb -- out[i] = sum_j coeffs[j] vecs[j][i] for 1 <= k <= 16 device
 * vectors of len FP64 values (coeffs and the pointer array on the host).
 * out may alias one of vecs.  Stream-ordered.  (Mixing and DIIS of the loop.)
 */
int thc_vec_lincomb(int k, const double *coeffs, const double *const *vecs, long long len, double *out,
                    void *stream);

#ifdef __cplusplus
}
#endif
#endif /* THC_DYSON_H */
