// Internal declarations of the THC self-energy library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "thc_sigma.h"

namespace thc {
// Kernel classes timed by the optional profiler (thc_profile / thc_profile_get).
enum KernelClass {
  K_UBUILD = 0,   // U_Pqs build
  K_PROJECT,      // X^T G(+-tau), G^X(+-tau)
  K_SOX_A,        // A_Pqv
  K_SOX_B,        // B_PRv
  K_SOX_CD,       // fused C_RvP and D_PR
  K_POLARISATION, // Pi = G^X(tau) o G^X(-tau)^T
  K_DIRECT_VPI,   // V Pi
  K_DIRECT_W,     // (V Pi) V with the merge epilogue
  K_BACK,         // M X^T and X (M X^T)
  K_ENERGY,       // trace and weighted sum
  K_SPLIT,        // FP64 <-> BF16 hi/lo conversions
  K_SOX_BCD,      // fused B_PRv and C/D (split precision)
  K_CHECK,        // non-finite input scans
  K_SCREEN,       // screened interaction of THC_GW: transforms and inversions
  K_COUNT
};
const char* kernel_class_name(int k);

struct ProfRec {
  int kclass;
  cudaEvent_t e0, e1;
  double flops;
};
struct ProfStat {
  long long launches = 0;
  double ms = 0.0, flops = 0.0;
};
}  // namespace thc

struct thc_ctx {
  int n = 0, N = 0, n_tau = 0;
  double beta = 0.0;
  int precision = THC_FP64, terms = THC_DIRECT | THC_SOX;
  cudaStream_t stream = nullptr;
  std::vector<double> tau;
  bool mirrored = false;  // tau_k + tau_{n_tau-1-k} == beta (within 1e-10 beta)

  // library-owned device memory
  double *X = nullptr, *V = nullptr;  // copies of the inputs
  double *U = nullptr;                // U_Pqs, N x n x n (FP64 path)
  // FP64 per-chunk workspace
  int tc = 1;   // tau points per chunk
  int Pb = 1;   // THC points per SOX block
  double *Y = nullptr, *Ym = nullptr;     // tc x N x n: X^T G(tau), X^T G(-tau)
  double *GXp = nullptr, *GXm = nullptr;  // tc x N x N: G^X(tau), G^X(-tau); GXm reused for V Pi
  double *Pi = nullptr;                   // tc x N x N: Pi, then reused for the merged M
  double *D = nullptr;                    // tc x N x N: D_PR
  double *T2 = nullptr;                   // tc x N x n: M X^T
  double *Ablk = nullptr;                 // Pb x n x n: A_Pqv for one P block
  double *Bblk = nullptr;                 // Pb x N x n: B_PRv for one P block
  // energy
  double *e_part = nullptr;   // n_tau partial traces
  double *e_w = nullptr;      // n_tau weights
  double *e_out = nullptr;    // 1 scalar
  // host-buffer entry point staging
  double *hG = nullptr, *hGb = nullptr, *hS = nullptr;

  // split-precision (THC_BF16X3) path: BF16 hi/lo pairs, leading dimensions padded to 8
  int ldn = 0, ldN = 0;                       // padded n and N
  // the constant operands X and V carry a third term (x = hi + lo + lo2 to about 24 bits)
  __nv_bfloat16 *Xt_h = nullptr, *Xt_l = nullptr, *Xt_l2 = nullptr;   // X^T, N x ldn
  __nv_bfloat16 *Xs_h = nullptr, *Xs_l = nullptr, *Xs_l2 = nullptr;   // X,   n x ldN
  __nv_bfloat16 *Vs_h = nullptr, *Vs_l = nullptr, *Vs_l2 = nullptr;   // V,   N x ldN
  __nv_bfloat16 *Us_h = nullptr, *Us_l = nullptr;   // U,   (N n) x ldn
  __nv_bfloat16 *Gs_h = nullptr, *Gs_l = nullptr;   // G(tau),  tc x n x ldn
  __nv_bfloat16 *Gms_h = nullptr, *Gms_l = nullptr; // G(-tau), tc x n x ldn
  __nv_bfloat16 *Ys_h = nullptr, *Ys_l = nullptr;   // X^T G(tau),  tc x N x ldn
  __nv_bfloat16 *Yms_h = nullptr, *Yms_l = nullptr; // X^T G(-tau), tc x N x ldn
  float *GXf = nullptr, *GXmf = nullptr;            // G^X(+-tau), tc x N x N
  __nv_bfloat16 *Pis_h = nullptr, *Pis_l = nullptr; // Pi,  tc x N x ldN
  __nv_bfloat16 *Ts_h = nullptr, *Ts_l = nullptr;   // V Pi, tc x N x ldN
  __nv_bfloat16 *Ms_h = nullptr, *Ms_l = nullptr;   // merged M, tc x N x ldN
  __nv_bfloat16 *T2s_h = nullptr, *T2s_l = nullptr; // (M X^T)^T, tc x n x ldN
  // third terms of the data operands of the direct chain and the back-transform (24 bits)
  __nv_bfloat16 *Gs_l2 = nullptr, *Gms_l2 = nullptr, *Ys_l2 = nullptr, *Yms_l2 = nullptr;
  __nv_bfloat16 *Pis_l2 = nullptr, *Ts_l2 = nullptr, *Ms_l2 = nullptr, *T2s_l2 = nullptr;
  __nv_bfloat16 *Ats_h = nullptr, *Ats_l = nullptr; // A^T blocks, Pb x n x ldn
  double *Dd = nullptr;                             // D, tc x N x N
  float *Pif = nullptr;                             // Pi of spin b, tc x N x N (unrestricted only)
  // screened direct term (THC_GW, FP64 path)
  int gw_nw = 0;                                    // sampled bosonic frequencies
  double *gw_toiw = nullptr, *gw_totau = nullptr;   // n_omega x n_tau, n_tau x n_omega
  double *gw_vinv = nullptr;                        // V^-1, N x N
  double *gw_pi = nullptr;                          // Pi~(tau), then W~(tau): n_tau x N x N
  double *gw_gx = nullptr;                          // G^X(tau), n_tau x N x N (restricted, or spin a)
  double *gw_gx_b = nullptr;                        // G^X(tau) of spin b (unrestricted, on first use)
  double *gw_w = nullptr;                           // W(i Omega), n_omega x N x N
  double *gw_scr = nullptr;                         // Gauss-Jordan scratch
  double *gw_m = nullptr;                           // split path: M of a chunk, tc x N x N
  size_t gw_scr_elems = 0;
  // device status words: [0] a tensor-core pipeline wait that ran out (its code),
  // [1] a non-finite value met in G_tau / G_bmt by an evaluation; read and cleared by status_check
  int *d_err = nullptr;

  std::vector<void*> owned;  // every cudaMalloc of this context
  std::string err;
  bool tuning = false;       // split path: time the tile widths of unseen contraction shapes

  // launch accounting and the optional profiler
  long long launch_count = 0;
  bool prof_on = false;
  std::vector<thc::ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  thc::ProfStat prof_stat[thc::K_COUNT];
};

namespace thc {

// Set-up that CUDA applies to one device (a kernel's shared-memory attribute, the
// SM count, the resident clusters of a launch shape): fn(dev, &value) runs once per
// (key, device) with that device current, under a lock; its value is cached and
// returned in *value.  A failing fn (non-zero return) caches nothing.
int per_device(const void* key, int* value, const std::function<int(int, int*)>& fn);

// Records msg on ctx and returns code.
int fail(thc_ctx* ctx, int code, const std::string& msg);
int check_cuda(thc_ctx* ctx, cudaError_t e, const char* what);
int ctx_alloc(thc_ctx* ctx, void** p, size_t bytes, const char* what);

// Bracket one kernel launch: call before the launch, then prof_end after it.
// Counts the launch; with the profiler on, records CUDA events on ctx->stream.
int prof_begin(thc_ctx* ctx, int kclass, double flops, thc::ProfRec* rec);
int prof_end(thc_ctx* ctx, thc::ProfRec* rec, cudaError_t launch_status, const char* what);
int prof_flush(thc_ctx* ctx);   // synchronises and folds pending events into the stats
void prof_release(thc_ctx* ctx);

// FP64 path (sigma_fp64.cu)
size_t fp64_workspace_bytes(int n, int N, int tc, int Pb);
int fp64_build_U(thc_ctx* ctx);
int fp64_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, double* Sigma);
// nspin = 1: restricted; nspin = 2: unrestricted spins a (index 0) and b (index 1)
int fp64_eval_spins(thc_ctx* ctx, int nspin, const double* const* G_tau, const double* const* G_bmt,
                    double* const* Sigma);
// D[b][P][R] = D[b][R][P] for P > R, b < batch (D_PR is symmetric; both paths compute P <= R)
int launch_mirror_upper(thc_ctx* ctx, double* D, long long N, long long batch);
int energy_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, const double* Sigma,
                const double* w_host, double* E);

// Context creation with an explicit workspace budget (0: a quarter of the free memory,
// or THC_WORKSPACE_BYTES); the batched API gives every molecule its own budget.
int ctx_create(thc_ctx** out, int n_ao, int n_thc, int n_tau, double beta, const double* X, const double* V,
               const double* tau, int precision, int terms, cudaStream_t stream, size_t budget);
void ctx_destroy(thc_ctx* ctx);

// screened direct term (gw.cu)
int gj_invert_spd(thc_ctx* ctx, double* A, long long n, long long batch);
int gw_set_transforms(thc_ctx* ctx, int n_omega, const double* to_iw, const double* to_tau);
int gw_store_bubble(thc_ctx* ctx, long long c0, long long tc, int nspin, int spin);
int gw_screen(thc_ctx* ctx);
int gw_merge(thc_ctx* ctx, long long c0, long long tc, const double* D, double* M, int spin);

// autotuner table of the split contractions (sigma_split.cu)
int autotune_save(const char* path);
int autotune_load(const char* path);
int autotune_entries();

// split-precision path (sigma_split.cu)
int split_init(thc_ctx* ctx, size_t budget);
int split_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, double* Sigma);
int split_eval_spins(thc_ctx* ctx, int nspin, const double* const* G_tau, const double* const* G_bmt,
                     double* const* Sigma);
// Synchronises and reads the status words: THC_ETIMEOUT if a tensor-core wait ran out,
// THC_EINVAL if an evaluation met a non-finite input; both are cleared.
int status_check(thc_ctx* ctx);
// Queues a scan of len FP64 values at p that sets d_err[1] if one is not finite.
int launch_finite_scan(thc_ctx* ctx, const double* p, long long len, int* flag);
int gemm_bf16x3(cudaStream_t stream, int batch, int M, int N, int K, const double* A, long long sA, const double* B,
                long long sB, double* C, long long sC);

}  // namespace thc

#define THC_TRY(...)           \
  do {                         \
    int _rc = (__VA_ARGS__);   \
    if (_rc != THC_OK) return _rc; \
  } while (0)
