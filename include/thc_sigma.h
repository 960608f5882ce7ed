/*
 * thc_sigma.h -- C ABI of the GB300 THC second-order self-energy library.
 *
 * The library evaluates the second-order self-energy of fully
 * self-consistent imaginary-time GF2 with tensor-hypercontracted (THC)
 * two-electron integrals (Pokhilko, Yeh, Morales, Zgid, arXiv:2404.17744):
 *
 *   Sigma(tau) = Sigma^dir(tau) + Sigma^SOX(tau)   at every tau point,
 *
 * with (pq|rs) = sum_PQ X_pP X_qP V_PQ X_rQ X_sQ (Eq. THC_ERI, the paper's
 * core matrix U_PQ is called V here).  SOX follows the paper's contraction
 * order (Sec. II.C): U_Pqs = sum_Q V_PQ X_qQ X_sQ built once, then per tau
 * the projections G_Rq, G_wP, the intermediates A_Pqv, B_PRv, C_RvP, D_PR
 * and the back-transform to Sigma_tr.  The direct term is the THC-GW form
 * of the second-order bubble (Sec. II.C, first paragraph):
 *   Pi = G^X(tau) o G^X(-tau),  W = V Pi V,  Sigma^dir = -2 X (G^X(tau) o W) X^T,
 * with G^X = X^T G X and o the elementwise product.
 *
 * Conventions shared by every entry point
 *   - All matrices are real, FP64, row-major.  G(tau) and Sigma(tau) are per
 *     spin (closed-shell restricted), symmetric n x n; the result for a
 *     non-symmetric G is unspecified.
 *   - G_pq(tau) = -<T p(tau) q^+> (Sec. II.A, Eq. G_def).  For 0 < tau < beta
 *     the library forms G(-tau) = -G(beta - tau).
 *   - Sign reading: the SOX term enters with +1 on G(-tau) (the paper prints
 *     -1, which matches if its "G(-tau)" denotes G(beta - tau)); the direct
 *     term carries -2 (closed spin loop).
 *   - "dev" pointers are CUDA device pointers owned by the caller; "host"
 *     pointers are ordinary host memory owned by the caller.  Everything the
 *     library allocates (U_Pqs, workspaces, copies of X and V) belongs to
 *     the context and is released by thc_destroy.
 *   - Calls are ordered on the context's stream and return before the GPU
 *     work finishes, except thc_energy and thc_sigma_eval_host, which
 *     synchronise the stream.
 *   - Return value: THC_OK (0) or a negative THC_E* code.  Nothing aborts,
 *     and no C++ exception crosses the ABI.  thc_last_error(ctx) describes
 *     the last failure on ctx (thc_last_error(NULL): the last failure of a
 *     thc_sigma_init on the calling thread).
 */
#ifndef THC_SIGMA_H
#define THC_SIGMA_H

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define THC_OK        0
#define THC_EINVAL   -1   /* bad sizes, NULL pointers, non-mirrored grid without G_bmt,
                             a NaN or infinite input value */
#define THC_ENOMEM   -2   /* device allocation failed */
#define THC_ECUDA    -3   /* a CUDA runtime call or kernel launch failed */
#define THC_ETIMEOUT -4   /* a bounded device-side wait ran out */
#define THC_ENOTSUP  -5   /* option not available in this build */

/* precision of the contractions */
#define THC_FP64     0    /* every step in FP64 (DFMA) */
#define THC_BF16X3   1    /* projections and V contractions as 3 BF16 products
                             (hi*hi + hi*lo + lo*hi) on tcgen05 tensor cores with
                             FP32 accumulation; inputs and outputs stay FP64 */
#define THC_TF32     2    /* not built: thc_sigma_init returns THC_ENOTSUP.  One TF32
                             product keeps 11 significant bits, too few for the 1e-6 Ha
                             bound on Sigma; three TF32 products meet it at half the
                             BF16 tensor rate, so THC_BF16X3 is the reduced-precision mode */

/* terms (bit mask) */
#define THC_DIRECT   1    /* second-order direct (bubble) term */
#define THC_SOX      2    /* second-order screened exchange */
#define THC_GW       4    /* screened direct term of scGW / scGWSOX (RPA W) in place of
                             THC_DIRECT (restricted, or unrestricted through
                             thc_sigma_eval_uhf); needs thc_sigma_set_bosonic */

typedef struct thc_ctx thc_ctx;   /* opaque, library-owned */

/*
 * thc_sigma_init -- set up a context and build U_Pqs = sum_Q V_PQ X_qQ X_sQ
 * (Eq. U_contraction, Sec. II.C: G-independent, built once, reused every
 * iteration).
 *   ctx       out: new context (NULL on failure)
 *   n_ao      n, number of atomic orbitals (>= 1)
 *   n_thc     N, number of THC interpolation points (>= 1)
 *   n_tau     number of imaginary-time points (>= 1)
 *   beta      inverse temperature (> 0)
 *   X         dev, n x N row-major collocation matrix X_iP (copied)
 *   V         dev, N x N row-major symmetric THC core (copied)
 *   tau       host, n_tau ascending points in (0, beta) (copied); if the grid
 *             is mirror-symmetric (|tau_k + tau_{n_tau-1-k} - beta| <= 1e-10 beta
 *             for all k) G(beta - tau_k) is read from G_tau itself
 *   precision THC_FP64 or THC_BF16X3 (THC_TF32: THC_ENOTSUP)
 *   terms     THC_DIRECT | THC_SOX, or THC_GW | THC_SOX (scGWSOX), non-zero;
 *             THC_DIRECT and THC_GW exclude each other
 *   stream    cudaStream_t the context launches on (NULL: legacy default stream)
 * X and V are scanned on the device: a NaN or infinite value gives THC_EINVAL.
 * Device memory held: U (N n^2 doubles) plus a workspace sized at init from
 * the free device memory (at most a quarter of it, or THC_WORKSPACE_BYTES
 * from the environment when set).
 */
int thc_sigma_init(thc_ctx **ctx, int n_ao, int n_thc, int n_tau, double beta,
                   const double *X, const double *V, const double *tau,
                   int precision, int terms, void *stream);

/*
 * thc_sigma_eval -- Sigma(tau_k) for every k (Sec. II.C scheme + direct term).
 *   G_tau      dev, n_tau x n x n, G(tau_k)
 *   G_bmt      dev, n_tau x n x n, G(beta - tau_k); NULL when the grid is
 *              mirror-symmetric (then G(beta - tau_k) = G_tau[n_tau-1-k])
 *   Sigma_tau  dev, n_tau x n x n, overwritten with Sigma(tau_k); must not
 *              alias G_tau or G_bmt
 * THC_EINVAL if G_bmt is NULL and the grid is not mirror-symmetric.  The call
 * stays asynchronous, so G is scanned for NaN and infinite values on the
 * stream and a hit is reported as THC_EINVAL by the next call that
 * synchronises (thc_sync, thc_energy, thc_sigma_eval_host, thc_sigma_tune).
 */
int thc_sigma_eval(thc_ctx *ctx, const double *G_tau, const double *G_bmt, double *Sigma_tau);

/*
 * thc_sigma_set_bosonic -- bosonic Matsubara transforms of the tau grid for the
 * screened direct term (THC_GW).  With the spin-summed THC polarisation
 * Pi~(tau) = 2 G^X(tau) o G^X(-tau)^T (G^X = X^T G X), evaluations compute
 *   Pi~(i W_m)  = sum_k to_iw[m][k] Pi~(tau_k),
 *   W(i W_m)    = V [1 - Pi~(i W_m) V]^{-1}   (formed as (V^{-1} - Pi~)^{-1}),
 *   W~(tau_k)   = sum_m to_tau[k][m] (W - V)(i W_m),
 *   Sigma^GW    = -X (G^X(tau) o W~(tau)) X^T     (Sec. II.C, THC-GW),
 * and add Sigma^SOX when THC_SOX is set (scGWSOX).  The first term of the series
 * W - V = V Pi~ V + ... is the THC_DIRECT term.
 *   n_omega  number of sampled bosonic frequencies (fixed once set)
 *   to_iw    host, n_omega x n_tau: values at the tau points -> values at i W_m
 *   to_tau   host, n_tau x n_omega: values at i W_m -> values at the tau points
 * Both map real functions symmetric under tau -> beta - tau (Pi~ and W~ of real
 * symmetric G); the frequencies need not be listed.  The first call allocates
 * 2 n_tau + n_omega + 1 N x N FP64 arrays (THC_BF16X3: tc more, the merged M of a tau
 * chunk) and inverts V on the device.  The transforms, the inversions (SPD, without
 * pivoting: Gauss-Jordan up to N = 128, above that the symmetric sweep in blocks of
 * 64 pivots on the upper triangle with DFMA trailing updates, N^3 flops) and the
 * merge run in FP64 on both paths; THC_BF16X3 takes G^X from its
 * split projections (FP32) and runs the back-transform on the tensor cores.
 * THC_EINVAL without THC_GW.  Synchronises.
 */
int thc_sigma_set_bosonic(thc_ctx *ctx, int n_omega, const double *to_iw, const double *to_tau);

/*
 * thc_sigma_eval_uhf -- spin-unrestricted Sigma_a(tau_k), Sigma_b(tau_k) for every k.
 * The paper writes the method for spin-orbitals (Sec. II.A); with spin-conserving
 * integrals and a G block-diagonal in spin, the second-order terms per spin s are
 *   Sigma^SOX_s: the Sec. II.C scheme with all three lines of spin s (+1), and
 *   Sigma^dir_s = -X (G^X_s(tau) o (V Pi V)) X^T with Pi summed over both spins,
 *                 Pi = sum_s' G^X_s'(tau) o G^X_s'(-tau)^T
 * (for G_a = G_b this is the restricted result of thc_sigma_eval for both spins).
 * With THC_GW the bubble is screened: Pi~ = sum_s' G^X_s'(tau) o G^X_s'(-tau)^T, one
 * W = V [1 - Pi~ V]^{-1} for both spins, Sigma^GW_s = -X (G^X_s o (W - V)) X^T; the
 * first unrestricted call allocates one more n_tau x N x N FP64 array (G^X of spin b).
 * The Galitskii-Migdal energy is one half of the sum over both spins of the
 * per-spin expression: E_dyn = (thc_energy(a) + thc_energy(b)) / 2.
 *   G_tau_a, G_tau_b    dev, n_tau x n x n, G of spin a and b
 *   G_bmt_a, G_bmt_b    dev G(beta - tau_k) of each spin, or NULL on a mirrored grid
 *   Sigma_a, Sigma_b    dev, n_tau x n x n, overwritten; distinct, aliasing no input
 * Same context (X, V, U, precision, terms) as the restricted evaluation; the split
 * path allocates one FP32 N x N buffer per tau chunk on its first unrestricted call.
 * Non-finite inputs are reported as for thc_sigma_eval.
 */
int thc_sigma_eval_uhf(thc_ctx *ctx, const double *G_tau_a, const double *G_bmt_a,
                       const double *G_tau_b, const double *G_bmt_b, double *Sigma_a,
                       double *Sigma_b);

/*
 * thc_sigma_eval_host -- thc_sigma_eval with host buffers: copies G in,
 * evaluates, copies Sigma out and synchronises.  The device staging buffers
 * are allocated on first use and kept by the context.  Pinned host memory
 * gives the fastest copies.  Arguments as for thc_sigma_eval, host pointers.
 */
int thc_sigma_eval_host(thc_ctx *ctx, const double *G_tau, const double *G_bmt, double *Sigma_tau);

/*
 * thc_energy -- Galitskii-Migdal dynamical energy on the tau axis (Eq. E2b):
 *   E_dyn = (1/beta) sum_n Tr[G(iw_n) Sigma(iw_n)]
 *         = -int_0^beta Tr[G(beta - tau) Sigma(tau)] dtau
 *        ~= -sum_k w_k Tr[G(beta - tau_k) Sigma(tau_k)],
 * per spin as written for the restricted G (spin sum and 1/2 cancel).
 *   G_tau, G_bmt  dev, as for thc_sigma_eval (G_bmt may be NULL on a mirrored grid)
 *   Sigma_tau     dev, n_tau x n x n
 *   tau_weights   host, n_tau quadrature weights of the tau grid
 *   E_dyn         host out
 * Reduction in FP64, fixed order (deterministic).  Synchronises the stream.
 */
int thc_energy(thc_ctx *ctx, const double *G_tau, const double *G_bmt,
               const double *Sigma_tau, const double *tau_weights, double *E_dyn);

/*
 * thc_sync -- wait for the work queued on ctx's stream and report what it met:
 * a tensor-core pipeline wait that ran out (THC_ETIMEOUT) or a NaN or infinite
 * value in an evaluation's G (THC_EINVAL).  Both reports are cleared.
 */
int thc_sync(thc_ctx *ctx);

/*
 * thc_gemm_bf16x3 -- C[b] = A[b] B[b]^T for FP64 matrices, computed as three
 * BF16 products (hi*hi + hi*lo + lo*hi, hi = bf16(x), lo = bf16(x - hi)) on
 * the tcgen05 tensor cores with FP32 accumulation: the contraction unit of
 * the THC_BF16X3 path (relative error about 1e-5 of sum_k |A_mk B_nk|).
 *   A  dev, batch x M x K row-major, consecutive batches strideA apart
 *      (strideA = 0: one A for every batch); B likewise N x K, strideB
 *   C  dev, batch x M x N row-major, strideC apart, overwritten
 *   stream  cudaStream_t (NULL: legacy default stream); synchronised
 * Temporary operand copies are allocated stream-ordered (cudaMallocAsync)
 * and freed before return.  Failures are described by thc_last_error(NULL).
 */
int thc_gemm_bf16x3(int batch, int M, int N, int K, const double *A, long long strideA,
                    const double *B, long long strideB, double *C, long long strideC, void *stream);

/*
 * thc_sigma_tune -- THC_BF16X3 contexts: run one evaluation on G_tau (dev;
 * G_bmt as for thc_sigma_eval) with the autotuner on, which times, for every
 * shape not yet in the table, both tensor-core tile widths of a single-chunk
 * contraction and the three cluster shapes (1 x 1, 1 x 2, 2 x 2 CTAs) of a
 * block of the fused B C/D kernel, and keeps the fastest; the evaluation's
 * output is discarded.  Later evaluations of any context use the table.
 * No-op for THC_FP64.  Synchronises.
 */
int thc_sigma_tune(thc_ctx *ctx, const double *G_tau, const double *G_bmt);

/* thc_autotune_save / thc_autotune_load -- write / merge the tile table
 * (text, one shape per line: class M N K batch choice, the choice being a tile
 * width 128 / 256, or 10 CP + CR for a fused B C/D block whose batch field is
 * its first P). */
int thc_autotune_save(const char *path);
int thc_autotune_load(const char *path);

/* thc_autotune_entries -- number of shapes in the tile table. */
int thc_autotune_entries(void);

/* thc_set_stream -- launch subsequent work of ctx on stream (cudaStream_t). */
int thc_set_stream(thc_ctx *ctx, void *stream);

/*
 * thc_sigma_flops -- algorithmic FP64-equivalent flop count of one
 * thc_sigma_eval on ctx (contractions only, 2 per multiply-add), for both terms:
 *   n_tau (2 N n^3 + 2 N (N + 1) n^2 + 4 N^3 + 6 N^2 n + N (N + 1) n + 6 N n^2),
 * and of the one-off U build, 2 N^2 n^2 (returned through u_flops if non-NULL).
 * The SOX intermediate D_PR is symmetric, so B, C and D are counted over the
 * N (N + 1) / 2 pairs P <= R that the library forms (the paper's scheme over all
 * (P, R) pairs would be 2 N^2 n^2 + N^2 n more per tau point).  With THC_GW the
 * count adds, per tau point, the projections (2 N n^2 + 4 N^2 n) and, per evaluation,
 * the two bosonic transforms (4 n_omega N^2 n_tau) and the n_omega inversions (N^3
 * each by the symmetric sweep above N = 128, 2 N^3 by Gauss-Jordan below).  The
 * profiler below reports what the kernels carry out, whole tiles included.
 */
double thc_sigma_flops(const thc_ctx *ctx, double *u_flops);

/*
 * thc_profile -- enable (1: clear counters and start) or stop (0) timing of
 * every kernel launch of ctx with CUDA events recorded on ctx's stream.
 * Timing adds two event records per launch; results are read with
 * thc_profile_get.  Synchronises the stream when pending events exist.
 */
int thc_profile(thc_ctx *ctx, int enable);

/*
 * thc_profile_get -- totals of kernel class kclass (0 <= kclass < number of
 * classes; THC_EINVAL past the last) since the last thc_profile(ctx, 1):
 * its name, number of launches, summed device time in ms and summed
 * flops those launches carried out (2 per multiply-add; for sox_B, sox_CD and
 * sox_BCD only the part of the (P, R) square they compute).  Any out-pointer
 * may be NULL.
 * Synchronises the stream.  Class names, by index from 0: u_build, project, sox_A, sox_B,
 * sox_CD, polarisation, direct_VPi, direct_W, back_transform, energy, split,
 * sox_BCD, check, screen (sox_B and sox_CD are the FP64 path's; the split path runs
 * both contractions as the one fused sox_BCD kernel; check is the non-finite input
 * scan; screen the bosonic transforms and inversions of THC_GW).
 */
int thc_profile_get(thc_ctx *ctx, int kclass, const char **name, long long *launches,
                    double *ms, double *flops);

/* thc_launch_count -- kernels launched by ctx since init (always counted). */
long long thc_launch_count(const thc_ctx *ctx);

/*
 * thc_energy_static -- the E_dyn of thc_energy for callers that cannot
 * allocate device memory (an external allocator owns the whole GPU, a plugin
 * may only use the buffers it is handed, or allocation is forbidden after
 * start-up).  The paper has no counterpart: this is a deployment variant.
 * It needs no context and calls no cudaMalloc/cudaFree; its scratch (partial
 * traces, weights, result) is a fixed device array of THC_STATIC_MAX_TAU
 * tau points that every GPU loading the library holds until exit.
 *   n_ao, n_tau   sizes; THC_EINVAL if n_tau > THC_STATIC_MAX_TAU
 *   G_tau, Sigma_tau  dev, n_tau x n_ao x n_ao
 *   G_bmt         dev G(beta - tau_k), or NULL to read G_tau[n_tau-1-k]
 *                 (the caller vouches that its grid is mirror-symmetric)
 *   tau_weights   host, n_tau quadrature weights
 *   E_dyn         host out; the result equals thc_energy's bit for bit
 *   stream        cudaStream_t (NULL: legacy default stream); synchronised
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  All calls share the array: calls that overlap
 * on the GPU (other streams or threads) race and must be serialised by the
 * caller.  Failures are described by thc_last_error(NULL).
 */
#define THC_STATIC_MAX_TAU 4096
int thc_energy_static(int n_ao, int n_tau, const double *G_tau, const double *G_bmt,
                      const double *Sigma_tau, const double *tau_weights, double *E_dyn,
                      void *stream);

/*
 * thc_wait_selftest -- exercises the failure path of the bounded device-side
 * waits (the paper has no counterpart: this checks the library's own error
 * handling).  One CTA holds TMEM and a bulk copy in flight, waits limit_ns on
 * an mbarrier that nothing ever completes, then unwinds as the tensor-core
 * kernels do after a timeout: it waits (bounded) for its copy and its
 * tensor-core operations, frees TMEM and returns.
 *   limit_ns  the wait's limit, 1e3 .. 1e9 ns (THC_EINVAL otherwise)
 *   stream    cudaStream_t (NULL: legacy default stream); synchronised
 * Returns THC_ETIMEOUT when the wait ran out and the unwind completed (the
 * expected result), THC_ECUDA if the unwind itself did not complete in time.
 * Allocates and frees 2 KB of device memory.  Failures are described by
 * thc_last_error(NULL).
 */
int thc_wait_selftest(long long limit_ns, void *stream);

/*
 * thc_fp64_dfma_rate -- measured FP64 peak of the current device: the rate of
 * independent fused multiply-adds (8 chains per thread, 4 CTAs of 256 threads
 * per SM, iters FMAs per chain), timed with CUDA events after one warm-up
 * launch.  GB300 has no FP64 tensor-core kind, so this DFMA rate bounds every
 * FP64 contraction of the library (the paper has no counterpart: it is the
 * denominator of the FP64 roofline).
 *   iters   FMAs per chain, 1 .. 2^40 (5e4 gives a launch of about 0.1 s on GB300)
 *   tflops  host out: 2 x FMAs / time / 1e12;  ms: host out (may be NULL)
 *   stream  cudaStream_t (NULL: legacy default stream); synchronised
 * Allocates and frees a few KB of device memory.
 */
int thc_fp64_dfma_rate(long long iters, double *tflops, double *ms, void *stream);

/* thc_destroy -- free everything ctx owns (NULL is a no-op).  Synchronises. */
void thc_destroy(thc_ctx *ctx);

/* thc_last_error -- text of the last failure on ctx, or of the last failed
 * init on this thread when ctx is NULL.  Never NULL; "" when none. */
const char *thc_last_error(const thc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* THC_SIGMA_H */
