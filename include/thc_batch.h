/*
 * thc_batch.h -- batched self-energy evaluation over many molecules.
 *
 * Evaluates Sigma(tau) = Sigma^dir + Sigma^SOX (thc_sigma.h, Sec. II.C of
 * arXiv:2404.17744) for n_mol independent molecules of uneven size on one GPU
 * in a single CUDA-graph launch.  The paper evaluates one molecule at a time
 * with MPI; this batching has no counterpart there.
 *
 * Molecule i has its own context (U_Pqs, blocking, workspace of at most
 * budget_per_molecule bytes; 0 = an equal share of a quarter of the free
 * memory, at least 64 MiB) bound to worker stream i % n_streams, so small
 * molecules run concurrently.  All molecules share one mirror-symmetric tau
 * grid (THC_EINVAL otherwise).  Return codes as in thc_sigma.h; failures are
 * described by thc_batch_last_error(b) or thc_last_error(NULL).
 */
#ifndef THC_BATCH_H
#define THC_BATCH_H

#include "thc_sigma.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thc_batch thc_batch;

/*
 * thc_batch_init -- n_ao[i], n_thc[i] sizes; X[i] (dev, n_ao x n_thc), V[i]
 * (dev, n_thc x n_thc) per molecule, copied; tau host (n_tau); precision as
 * in thc_sigma_init; tune != 0 turns the tensor-core autotuner on for the
 * first evaluation; stream: the stream graph launches are ordered on.
 */
int thc_batch_init(thc_batch **b, int n_mol, const int *n_ao, const int *n_thc, int n_tau, double beta,
                   const double *const *X, const double *const *V, const double *tau, int precision,
                   int n_streams, unsigned long long budget_per_molecule, int tune, void *stream);

/*
 * thc_batch_eval -- Sigma_tau[i] (dev, n_tau x n_ao[i] x n_ao[i]) from
 * G_tau[i] (dev) for every molecule; the pointer arrays are host arrays.
 * The first call with a given set of buffers runs every molecule once (and
 * tunes), then captures the whole batch into a CUDA graph and launches it;
 * later calls with the same buffers only launch the graph.  Stream-ordered
 * on the batch's stream.
 */
int thc_batch_eval(thc_batch *b, const double *const *G_tau, double *const *Sigma_tau);

/* thc_batch_graph_info -- kernels in the captured graph and its node count. */
int thc_batch_graph_info(const thc_batch *b, long long *kernel_launches, long long *graph_nodes);

/* thc_batch_flops -- algorithmic flops of one batched evaluation (sum of thc_sigma_flops). */
double thc_batch_flops(const thc_batch *b);

const char *thc_batch_last_error(const thc_batch *b);
void thc_batch_destroy(thc_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* THC_BATCH_H */
