/*
 * thc_learned.h -- learned self-energy proposals for the self-consistency loop.
 *
 * The paper (arXiv:2404.17744) iterates Sigma[G] and the Dyson equation to
 * full self-consistency with damping and DIIS (Sec. III.A); it has no learned
 * component.  These entry points add one that cannot change the fixed point:
 * a proposal is only an input self-energy, and the exact Sigma evaluation of
 * the next iteration judges it (the loop driver keeps it only if the residual
 * improves).
 *
 * Network: a two-layer perceptron shared by all matrix elements e,
 *     y = W2 relu(W1 x + b1) + b2,   x in R^{d_in}, y in R^{d_out},
 * FP16 working weights, FP32 master weights, FP32 accumulation, Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8), mean-squared-error loss
 * (1 / (B d_out)) sum (y - t)^2 over a batch of B samples.  All arrays are
 * row-major FP32: X is B x d_in, T and Y are B x d_out, W1 is hidden x d_in,
 * W2 is d_out x hidden.  Return codes as in thc_sigma.h.
 */
#ifndef THC_LEARNED_H
#define THC_LEARNED_H

#include <stddef.h>

#include "thc_sigma.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thc_mlp thc_mlp;
typedef struct thc_proposer thc_proposer;

/* thc_mlp_init -- network with the given initial weights (host or dev, FP32,
 * copied); max_batch bounds every later batch. */
int thc_mlp_init(thc_mlp **m, int d_in, int hidden, int d_out, int max_batch, const float *W1,
                 const float *b1, const float *W2, const float *b2, void *stream);

/* thc_mlp_forward -- Y (dev, batch x d_out) = network(X (dev, batch x d_in)). */
int thc_mlp_forward(thc_mlp *m, int batch, const float *X, float *Y);

/* thc_mlp_gradients -- loss and its gradients with respect to W1, b1, W2, b2 for
 * the batch (X, T); outputs host or dev, any may be NULL.  Synchronises. */
int thc_mlp_gradients(thc_mlp *m, int batch, const float *X, const float *T, double *loss, float *gW1,
                      float *gb1, float *gW2, float *gb2);

/* thc_mlp_train -- `steps` Adam steps on n_samples (X, T), mini-batches of
 * min(batch, n_samples, max_batch) samples in a fixed cyclic order; final_loss
 * (host, may be NULL) is the loss of the last mini-batch before its update. */
int thc_mlp_train(thc_mlp *m, int n_samples, const float *X, const float *T, int steps, int batch,
                  double lr, double *final_loss);

/* thc_mlp_get_weights -- copy the FP32 master weights out (host or dev; NULL skips). */
int thc_mlp_get_weights(thc_mlp *m, float *W1, float *b1, float *W2, float *b2);

void thc_mlp_destroy(thc_mlp *m);

/*
 * thc_proposer_init -- proposer over the IR coefficients of Sigma:
 *   c_k = fit_tau Sigma_k(tau)  (n_l x n_ao^2),
 *   inputs x_e = [c_k[:, e] / s_c, (c_k - c_{k-1})[:, e] / s_d]  (d_in = 2 n_l),
 *   proposal c = c_k + s_d MLP(x_e)  (d_out = n_l), returned as Sigma(tau) = U_tau c,
 * with s_c, s_d the root-mean-square of c_k and of c_k - c_{k-1}.  Training
 * pairs: (x built from c_j and c_{j-1}) -> (c_latest - c_j) / s_d(j) for the
 * observed iterates j inside the history window max_hist (>= 3), each scaled by
 * the RMS s_d(j) of its own change c_j - c_{j-1} and s_c of the latest iterate.
 *   U_tau host n_tau x n_l, fit_tau host n_l x n_tau (the IR sampling matrices);
 *   W1 (hidden x 2 n_l), b1, W2 (n_l x hidden), b2: initial weights, host FP32.
 */
int thc_proposer_init(thc_proposer **p, int n_ao, int n_tau, int n_l, const double *U_tau,
                      const double *fit_tau, int hidden, int max_hist, const float *W1, const float *b1,
                      const float *W2, const float *b2, void *stream);

/* thc_proposer_observe -- record the exact Sigma(tau) (dev) of the latest iteration. */
int thc_proposer_observe(thc_proposer *p, const double *Sigma_tau);

/* thc_proposer_count -- number of iterates observed. */
int thc_proposer_count(const thc_proposer *p);

/* thc_proposer_reset -- forget the observed trajectory, keep the trained
 * network: a network fitted on one run's trajectory can then propose for
 * another run of the same sizes (transfer between related systems). */
int thc_proposer_reset(thc_proposer *p);

/* thc_proposer_train -- build the training pairs from the window and run
 * `steps` Adam steps (mini-batch `batch`); needs >= 3 observed iterates. */
int thc_proposer_train(thc_proposer *p, int steps, int batch, double lr, double *final_loss);

/* thc_proposer_propose -- write the proposed Sigma(tau) (dev, n_tau x n_ao x n_ao)
 * from the last two observed iterates (s_c, s_d taken from them).  Synchronises. */
int thc_proposer_propose(thc_proposer *p, double *Sigma_tau);

/* Resumable state of a proposer (checkpoint / resume of a self-consistent run):
 * a header (sizes, observed-iterate count, Adam step, the scales s_c and s_d),
 * the FP32 master weights and Adam moments of the network, and the observed
 * coefficient window (the last min(count, max_hist) iterates, FP64).  The FP16
 * working copies are rebuilt from the masters on load.
 *
 * thc_proposer_state_size -- bytes of the current state into *bytes.
 * thc_proposer_save_state -- copy the state into the host buffer buf of `bytes`
 *   bytes (>= the size; THC_EINVAL otherwise).  Synchronises.
 * thc_proposer_load_state -- restore a state saved by a proposer of the same
 *   n_ao, n_tau, n_l, hidden and max_hist; THC_EINVAL on any mismatch or a short
 *   buffer (the proposer is then left unchanged).  Synchronises. */
int thc_proposer_state_size(const thc_proposer *p, size_t *bytes);
int thc_proposer_save_state(thc_proposer *p, void *buf, size_t bytes);
int thc_proposer_load_state(thc_proposer *p, const void *buf, size_t bytes);

const char *thc_proposer_last_error(const thc_proposer *p);
void thc_proposer_destroy(thc_proposer *p);

#ifdef __cplusplus
}
#endif
#endif /* THC_LEARNED_H */
