// C ABI of the THC self-energy library (declared in include/thc_sigma.h).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>

#include "thc_internal.cuh"

namespace {
thread_local std::string g_init_error;
}  // namespace

namespace thc {

int per_device(const void* key, int* value, const std::function<int(int, int*)>& fn) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return THC_ECUDA;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({key, dev});
  if (it != cache.end()) {
    if (value) *value = it->second;
    return THC_OK;
  }
  int v = 0;
  const int rc = fn(dev, &v);
  if (rc != THC_OK) return rc;
  cache[{key, dev}] = v;
  if (value) *value = v;
  return THC_OK;
}

namespace {
// flag <- 1 if any of the len values at p is NaN or infinite (grid-stride, no atomics on the
// common path: a warp votes and one lane writes).
__global__ void finite_scan_kernel(const double* __restrict__ p, long long len, int* flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}
}  // namespace

int launch_finite_scan(thc_ctx* ctx, const double* p, long long len, int* flag) {
  if (len <= 0) return THC_OK;
  const int blocks = (int)std::min<long long>((len + 255) / 256, 152LL * 8);
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_CHECK, 0.0, &rec));
  finite_scan_kernel<<<blocks, 256, 0, ctx->stream>>>(p, len, flag);
  return prof_end(ctx, &rec, cudaGetLastError(), "non-finite input scan");
}

int status_check(thc_ctx* ctx) {
  if (!ctx->d_err) return THC_OK;
  int h[2] = {0, 0};
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream),
                     "read status words"));
  THC_TRY(check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "status sync"));
  if (h[0] || h[1]) {
    THC_TRY(check_cuda(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(h), ctx->stream), "clear status words"));
    if (h[0]) return fail(ctx, THC_ETIMEOUT, "a tensor-core pipeline wait ran out (code " + std::to_string(h[0]) + ")");
    return fail(ctx, THC_EINVAL, "G_tau or G_bmt held a NaN or infinite value (met by an evaluation since the "
                                 "last synchronising call); the Sigma it produced is not valid");
  }
  return THC_OK;
}

int fail(thc_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_init_error = msg;
  return code;
}

int check_cuda(thc_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return THC_OK;
  const int code = (e == cudaErrorMemoryAllocation) ? THC_ENOMEM : THC_ECUDA;
  return fail(ctx, code, std::string(what) + ": " + cudaGetErrorString(e));
}

int ctx_alloc(thc_ctx* ctx, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) return THC_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    *p = nullptr;
    return fail(ctx, THC_ENOMEM, std::string("cudaMalloc ") + what + " (" + std::to_string(bytes) + " bytes): " +
                                     cudaGetErrorString(e));
  }
  ctx->owned.push_back(*p);
  return THC_OK;
}

}  // namespace thc

namespace {

void release(thc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  thc::prof_release(ctx);
  for (void* p : ctx->owned) cudaFree(p);
  ctx->owned.clear();
}

// budget 0 -> THC_WORKSPACE_BYTES if set, else a quarter of the free device memory
int default_budget(thc_ctx* ctx, size_t* budget) {
  if (*budget > 0) return THC_OK;
  if (const char* env = std::getenv("THC_WORKSPACE_BYTES")) {
    const unsigned long long v = std::strtoull(env, nullptr, 10);
    if (v > 0) {
      *budget = (size_t)v;
      return THC_OK;
    }
  }
  size_t free_b = 0, total_b = 0;
  THC_TRY(thc::check_cuda(ctx, cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo"));
  *budget = free_b / 4;
  return THC_OK;
}

int choose_blocking(thc_ctx* ctx, size_t budget) {
  const size_t d = sizeof(double);
  const size_t n = ctx->n, N = ctx->N;
  const size_t per_p = d * (n * n + N * n);
  const size_t per_t = d * (3 * N * n + 4 * N * N);
  size_t pb = std::max<size_t>(1, (budget / 2) / per_p);
  pb = std::min<size_t>(pb, N);
  size_t rest = budget > pb * per_p ? budget - pb * per_p : 0;
  size_t tc = std::max<size_t>(1, rest / per_t);
  tc = std::min<size_t>(tc, (size_t)ctx->n_tau);
  ctx->Pb = (int)pb;
  ctx->tc = (int)tc;
  return THC_OK;
}

int init_impl(thc_ctx* ctx, const double* X, const double* V, const double* tau, size_t budget_in) {
  using namespace thc;
  const size_t n = ctx->n, N = ctx->N, nt = ctx->n_tau;
  ctx->tau.assign(tau, tau + nt);
  for (size_t k = 0; k < nt; ++k) {
    if (!(tau[k] > 0.0 && tau[k] < ctx->beta) || (k > 0 && !(tau[k] > tau[k - 1])))
      return fail(ctx, THC_EINVAL, "tau must be strictly ascending inside (0, beta)");
  }
  ctx->mirrored = true;
  for (size_t k = 0; k < nt; ++k)
    if (std::fabs(tau[k] + tau[nt - 1 - k] - ctx->beta) > 1e-10 * ctx->beta) ctx->mirrored = false;

  THC_TRY(ctx_alloc(ctx, (void**)&ctx->X, sizeof(double) * n * N, "X"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->V, sizeof(double) * N * N, "V"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->d_err, 2 * sizeof(int), "status words"));
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->X, X, sizeof(double) * n * N, cudaMemcpyDefault, ctx->stream), "copy X"));
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->V, V, sizeof(double) * N * N, cudaMemcpyDefault, ctx->stream), "copy V"));
  {  // X and V must be finite: checked here, synchronously, with the status word of G
    int* flag = ctx->d_err + 1;
    int h = 0;
    THC_TRY(check_cuda(ctx, cudaMemsetAsync(ctx->d_err, 0, 2 * sizeof(int), ctx->stream), "clear status words"));
    THC_TRY(launch_finite_scan(ctx, ctx->X, (long long)(n * N), flag));
    THC_TRY(launch_finite_scan(ctx, ctx->V, (long long)(N * N), flag));
    THC_TRY(check_cuda(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "read flag"));
    THC_TRY(check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "input check sync"));
    if (h) return fail(ctx, THC_EINVAL, "X or V holds a NaN or infinite value");
  }
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->e_part, sizeof(double) * nt, "energy partials"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->e_w, sizeof(double) * nt, "energy weights"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->e_out, sizeof(double), "energy"));

  if (ctx->precision == THC_FP64) {
    if (ctx->terms & THC_SOX) THC_TRY(ctx_alloc(ctx, (void**)&ctx->U, sizeof(double) * N * n * n, "U"));
    size_t free_b = 0, total_b = 0;
    THC_TRY(check_cuda(ctx, cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo"));
    size_t budget = free_b / 4;
    if (const char* env = std::getenv("THC_WORKSPACE_BYTES")) {
      const unsigned long long v = std::strtoull(env, nullptr, 10);
      if (v > 0) budget = (size_t)v;
    }
    choose_blocking(ctx, budget);
    const size_t NN = N * N, Nn = N * n, tc = ctx->tc, pb = ctx->Pb;
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->Y, sizeof(double) * tc * Nn, "Y"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->Ym, sizeof(double) * tc * Nn, "Ym"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->GXp, sizeof(double) * tc * NN, "GX+"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->GXm, sizeof(double) * tc * NN, "GX-"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->Pi, sizeof(double) * tc * NN, "Pi"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->D, sizeof(double) * tc * NN, "D"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->T2, sizeof(double) * tc * Nn, "T2"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->Ablk, sizeof(double) * pb * n * n, "A block"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->Bblk, sizeof(double) * pb * Nn, "B block"));
    if (ctx->terms & THC_SOX) THC_TRY(fp64_build_U(ctx));
  } else {
    size_t budget = budget_in;
    THC_TRY(default_budget(ctx, &budget));
    THC_TRY(split_init(ctx, budget));
  }
  return THC_OK;
}

}  // namespace

namespace thc {

int ctx_create(thc_ctx** out, int n_ao, int n_thc, int n_tau, double beta, const double* X, const double* V,
               const double* tau, int precision, int terms, cudaStream_t stream, size_t budget) {
  *out = nullptr;
  if (n_ao < 1 || n_thc < 1 || n_tau < 1 || !(beta > 0.0))
    return fail(nullptr, THC_EINVAL, "need n_ao, n_thc, n_tau >= 1 and beta > 0");
  if (n_thc > 65535) return fail(nullptr, THC_EINVAL, "n_thc above 65535 is not supported");
  if (!X || !V || !tau) return fail(nullptr, THC_EINVAL, "X, V and tau must be non-NULL");
  if (precision == THC_TF32)
    return fail(nullptr, THC_ENOTSUP,
                "THC_TF32 is not built: one TF32 product (11 significant bits) misses the 1e-6 Ha bound on "
                "Sigma, and three TF32 products run at half the BF16 tensor rate for the bound THC_BF16X3 meets");
  if (precision != THC_FP64 && precision != THC_BF16X3) return fail(nullptr, THC_EINVAL, "unknown precision");
  if (terms <= 0 || terms > (THC_DIRECT | THC_SOX | THC_GW) || ((terms & THC_DIRECT) && (terms & THC_GW)))
    return fail(nullptr, THC_EINVAL, "terms must be THC_DIRECT and/or THC_SOX, or THC_GW with or without THC_SOX");
  thc_ctx* ctx = nullptr;
  try {
    ctx = new thc_ctx();
  } catch (...) {
    return fail(nullptr, THC_ENOMEM, "host allocation of the context failed");
  }
  ctx->n = n_ao;
  ctx->N = n_thc;
  ctx->n_tau = n_tau;
  ctx->beta = beta;
  ctx->precision = precision;
  ctx->terms = terms;
  ctx->stream = stream;
  int rc;
  try {
    rc = init_impl(ctx, X, V, tau, budget);
  } catch (...) {
    rc = fail(ctx, THC_ENOMEM, "host allocation failed during init");
  }
  if (rc != THC_OK) {
    g_init_error = ctx->err;
    release(ctx);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return THC_OK;
}

void ctx_destroy(thc_ctx* ctx) {
  if (!ctx) return;
  release(ctx);
  delete ctx;
}

}  // namespace thc

extern "C" {

int thc_sigma_init(thc_ctx** out, int n_ao, int n_thc, int n_tau, double beta, const double* X, const double* V,
                   const double* tau, int precision, int terms, void* stream) {
  g_init_error.clear();
  if (!out) return thc::fail(nullptr, THC_EINVAL, "ctx out-pointer is NULL");
  return thc::ctx_create(out, n_ao, n_thc, n_tau, beta, X, V, tau, precision, terms, (cudaStream_t)stream, 0);
}

int thc_sigma_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, double* Sigma_tau) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  if (!G_tau || !Sigma_tau) return fail(ctx, THC_EINVAL, "G_tau and Sigma_tau must be non-NULL");
  if (!G_bmt && !ctx->mirrored) return fail(ctx, THC_EINVAL, "tau grid is not mirror-symmetric: pass G_bmt");
  if (Sigma_tau == G_tau || (G_bmt && Sigma_tau == G_bmt)) return fail(ctx, THC_EINVAL, "Sigma_tau aliases an input");
  const long long len = (long long)ctx->n_tau * ctx->n * ctx->n;
  THC_TRY(launch_finite_scan(ctx, G_tau, len, ctx->d_err + 1));
  if (G_bmt) THC_TRY(launch_finite_scan(ctx, G_bmt, len, ctx->d_err + 1));
  try {
    if (ctx->precision == THC_FP64) return fp64_eval(ctx, G_tau, G_bmt, Sigma_tau);
    return split_eval(ctx, G_tau, G_bmt, Sigma_tau);
  } catch (...) {
    return fail(ctx, THC_ENOMEM, "host allocation failed during eval");
  }
}

int thc_sigma_eval_uhf(thc_ctx* ctx, const double* G_tau_a, const double* G_bmt_a, const double* G_tau_b,
                       const double* G_bmt_b, double* Sigma_a, double* Sigma_b) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  if (!G_tau_a || !G_tau_b || !Sigma_a || !Sigma_b) return fail(ctx, THC_EINVAL, "NULL argument to thc_sigma_eval_uhf");
  if ((!G_bmt_a || !G_bmt_b) && !ctx->mirrored)
    return fail(ctx, THC_EINVAL, "tau grid is not mirror-symmetric: pass G_bmt for both spins");
  const double* in[4] = {G_tau_a, G_bmt_a, G_tau_b, G_bmt_b};
  for (const double* p : in)
    if (p && (p == Sigma_a || p == Sigma_b)) return fail(ctx, THC_EINVAL, "a Sigma output aliases an input");
  if (Sigma_a == Sigma_b) return fail(ctx, THC_EINVAL, "Sigma_a and Sigma_b must differ");
  const long long len = (long long)ctx->n_tau * ctx->n * ctx->n;
  for (const double* p : in)
    if (p) THC_TRY(launch_finite_scan(ctx, p, len, ctx->d_err + 1));
  const double* G[2] = {G_tau_a, G_tau_b};
  const double* Gb[2] = {G_bmt_a, G_bmt_b};
  double* S[2] = {Sigma_a, Sigma_b};
  try {
    if (ctx->precision == THC_FP64) return fp64_eval_spins(ctx, 2, G, Gb, S);
    return split_eval_spins(ctx, 2, G, Gb, S);
  } catch (...) {
    return fail(ctx, THC_ENOMEM, "host allocation failed during eval");
  }
}

int thc_sigma_eval_host(thc_ctx* ctx, const double* G_tau, const double* G_bmt, double* Sigma_tau) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  if (!G_tau || !Sigma_tau) return fail(ctx, THC_EINVAL, "G_tau and Sigma_tau must be non-NULL");
  const size_t bytes = sizeof(double) * (size_t)ctx->n_tau * ctx->n * ctx->n;
  if (!ctx->hG) THC_TRY(ctx_alloc(ctx, (void**)&ctx->hG, bytes, "host-entry G"));
  if (!ctx->hS) THC_TRY(ctx_alloc(ctx, (void**)&ctx->hS, bytes, "host-entry Sigma"));
  if (G_bmt && !ctx->hGb) THC_TRY(ctx_alloc(ctx, (void**)&ctx->hGb, bytes, "host-entry G(beta-tau)"));
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->hG, G_tau, bytes, cudaMemcpyHostToDevice, ctx->stream), "H2D G"));
  if (G_bmt)
    THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->hGb, G_bmt, bytes, cudaMemcpyHostToDevice, ctx->stream), "H2D Gb"));
  THC_TRY(thc_sigma_eval(ctx, ctx->hG, G_bmt ? ctx->hGb : nullptr, ctx->hS));
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(Sigma_tau, ctx->hS, bytes, cudaMemcpyDeviceToHost, ctx->stream), "D2H Sigma"));
  THC_TRY(check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "host-entry sync"));
  return status_check(ctx);
}

int thc_energy(thc_ctx* ctx, const double* G_tau, const double* G_bmt, const double* Sigma_tau,
               const double* tau_weights, double* E_dyn) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  if (!G_tau || !Sigma_tau || !tau_weights || !E_dyn) return fail(ctx, THC_EINVAL, "NULL argument to thc_energy");
  if (!G_bmt && !ctx->mirrored) return fail(ctx, THC_EINVAL, "tau grid is not mirror-symmetric: pass G_bmt");
  THC_TRY(energy_eval(ctx, G_tau, G_bmt, Sigma_tau, tau_weights, E_dyn));
  return status_check(ctx);
}

int thc_sync(thc_ctx* ctx) {
  if (!ctx) return thc::fail(nullptr, THC_EINVAL, "ctx is NULL");
  THC_TRY(thc::check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync"));
  return thc::status_check(ctx);
}

int thc_gemm_bf16x3(int batch, int M, int N, int K, const double* A, long long strideA, const double* B,
                    long long strideB, double* C, long long strideC, void* stream) {
  using namespace thc;
  if (batch < 1 || M < 1 || N < 1 || K < 1 || batch > 65535)
    return fail(nullptr, THC_EINVAL, "thc_gemm_bf16x3: need 1 <= batch <= 65535 and M, N, K >= 1");
  if (!A || !B || !C) return fail(nullptr, THC_EINVAL, "thc_gemm_bf16x3: NULL operand");
  if (strideA < 0 || strideB < 0 || (batch > 1 && strideC < (long long)M * N))
    return fail(nullptr, THC_EINVAL, "thc_gemm_bf16x3: bad batch strides");
  try {
    return gemm_bf16x3((cudaStream_t)stream, batch, M, N, K, A, strideA, B, strideB, C, strideC);
  } catch (...) {
    return fail(nullptr, THC_ENOMEM, "thc_gemm_bf16x3: host allocation failed");
  }
}

int thc_set_stream(thc_ctx* ctx, void* stream) {
  if (!ctx) return thc::fail(nullptr, THC_EINVAL, "ctx is NULL");
  ctx->stream = (cudaStream_t)stream;
  return THC_OK;
}

double thc_sigma_flops(const thc_ctx* ctx, double* u_flops) {
  if (!ctx) return 0.0;
  const double n = ctx->n, N = ctx->N, nt = ctx->n_tau;
  double f = 4.0 * N * n * n + 2.0 * N * N * n;  // Y, M X^T, X T2
  // SOX: A for all P, then B and C/D for the N (N + 1) / 2 pairs P <= R (D_PR is symmetric)
  if (ctx->terms & THC_SOX) f += 2.0 * N * n * n * n + 2.0 * N * (N + 1) * n * n + N * (N + 1) * n;
  if (ctx->terms & THC_DIRECT) f += 2.0 * N * n * n + 4.0 * N * N * n + 4.0 * N * N * N;
  if (ctx->terms & THC_GW) {  // projections per tau; per evaluation the transforms and the inversions
    // (the symmetric sweep above 128 rows: N^3 each; Gauss-Jordan on the whole matrix below: 2 N^3)
    const double nw = ctx->gw_nw, inv = (ctx->N > 128 ? 1.0 : 2.0) * N * N * N;
    f += 2.0 * N * n * n + 4.0 * N * N * n;
    if (nt > 0) f += (4.0 * nw * N * N * nt + nw * inv) / nt;
  }
  if (u_flops) *u_flops = (ctx->terms & THC_SOX) ? 2.0 * N * N * n * n : 0.0;
  return nt * f;
}

int thc_profile(thc_ctx* ctx, int enable) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  THC_TRY(prof_flush(ctx));
  if (enable)
    for (int k = 0; k < K_COUNT; ++k) ctx->prof_stat[k] = ProfStat();
  ctx->prof_on = enable != 0;
  return THC_OK;
}

int thc_profile_get(thc_ctx* ctx, int kclass, const char** name, long long* launches, double* ms, double* flops) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  if (kclass < 0 || kclass >= K_COUNT) return THC_EINVAL;
  THC_TRY(prof_flush(ctx));
  if (name) *name = kernel_class_name(kclass);
  if (launches) *launches = ctx->prof_stat[kclass].launches;
  if (ms) *ms = ctx->prof_stat[kclass].ms;
  if (flops) *flops = ctx->prof_stat[kclass].flops;
  return THC_OK;
}

long long thc_launch_count(const thc_ctx* ctx) { return ctx ? ctx->launch_count : 0; }

void thc_destroy(thc_ctx* ctx) { thc::ctx_destroy(ctx); }

int thc_sigma_tune(thc_ctx* ctx, const double* G_tau, const double* G_bmt) {
  using namespace thc;
  if (!ctx) return fail(nullptr, THC_EINVAL, "ctx is NULL");
  if (!G_tau) return fail(ctx, THC_EINVAL, "G_tau must be non-NULL");
  if (ctx->precision != THC_BF16X3) return THC_OK;  // the FP64 path has one tile shape
  const size_t bytes = sizeof(double) * (size_t)ctx->n_tau * ctx->n * ctx->n;
  if (!ctx->hS) THC_TRY(ctx_alloc(ctx, (void**)&ctx->hS, bytes, "tuning output"));
  ctx->tuning = true;
  int rc = thc_sigma_eval(ctx, G_tau, G_bmt, ctx->hS);
  ctx->tuning = false;
  THC_TRY(rc);
  return thc_sync(ctx);
}

int thc_autotune_save(const char* path) {
  if (!path) return thc::fail(nullptr, THC_EINVAL, "thc_autotune_save: NULL path");
  return thc::autotune_save(path);
}

int thc_autotune_load(const char* path) {
  if (!path) return thc::fail(nullptr, THC_EINVAL, "thc_autotune_load: NULL path");
  return thc::autotune_load(path);
}

int thc_autotune_entries(void) { return thc::autotune_entries(); }

const char* thc_last_error(const thc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

}  // extern "C"
