// Screened direct term (scGW, scGWSOX; Sec. II.C, first paragraph: the THC-GW
// scheme) on the FP64 path.  Restricted, per spin:
//
//   Pi~(tau)   = 2 G^X(tau) o G^X(-tau)^T                   (spin-summed bubble)
//   Pi~(i W_m) = sum_k to_iw[m][k] Pi~(tau_k)                (bosonic transform)
//   W(i W_m)   = V [1 - Pi~ V]^{-1} = (V^{-1} - Pi~)^{-1}    (SPD: V SPD, Pi~ <= 0)
//   W~(tau_k)  = sum_m to_tau[k][m] (W - V)(i W_m)
//   Sigma^GW   = -X (G^X(tau) o W~(tau)) X^T
//
// W is formed as the inverse of the symmetric positive definite V^{-1} - Pi~, a
// Gauss-Jordan elimination without pivoting (stable for SPD matrices), batched
// over the sampled frequencies; V^{-1} is formed the same way once per context.
// The transforms to_iw, to_tau are inputs (the bosonic sampling matrices of the
// caller's tau grid).  All arithmetic is FP64 in the DFMA tile or plain kernels.
#include <algorithm>

#include "dfma_tile.cuh"
#include "thc_internal.cuh"

namespace thc {
namespace {

using f64::View;

int blocks_for(long long total) { return (int)std::min<long long>((total + 255) / 256, 152LL * 32); }

// Step k of the in-place Gauss-Jordan inverse of B matrices (n x n, contiguous):
// save row k, column k and 1 / a_kk of every matrix ...
__global__ void gj_pivot_kernel(long long n, int k, double* __restrict__ A, double* __restrict__ row,
                                double* __restrict__ col, double* __restrict__ piv) {
  const long long b = blockIdx.x, nn = n * n;
  const double* a = A + b * nn;
  for (long long j = threadIdx.x; j < n; j += blockDim.x) {
    row[b * n + j] = a[(long long)k * n + j];
    col[b * n + j] = a[j * n + k];
  }
  if (threadIdx.x == 0) piv[b] = 1.0 / a[(long long)k * n + k];
}

// ... then a_kk <- p, a_kj <- a_kj p, a_ik <- -a_ik p, a_ij <- a_ij - a_ik a_kj p (p = 1 / a_kk).
__global__ void gj_update_kernel(long long n, int k, long long batch, double* __restrict__ A,
                                 const double* __restrict__ row, const double* __restrict__ col,
                                 const double* __restrict__ piv) {
  const long long nn = n * n, total = nn * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / nn, e = idx - b * nn, i = e / n, j = e - i * n;
    const double p = piv[b];
    double v;
    if (i == k)
      v = (j == k) ? p : row[b * n + j] * p;
    else if (j == k)
      v = -col[b * n + i] * p;
    else
      v = fma(-col[b * n + i] * p, row[b * n + j], A[idx]);
    A[idx] = v;
  }
}

// Pi~[k0 + b] = 2 GXp[b] o GXm[b]^T and GX[k0 + b] = GXp[b] for the tau points of a chunk.
__global__ void gw_bubble_kernel(long long N, long long batch, const double* __restrict__ GXp,
                                 const double* __restrict__ GXm, double* __restrict__ Pi, double* __restrict__ GX) {
  const long long NN = N * N, total = NN * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / NN, r = idx - b * NN, i = r / N, j = r - i * N;
    Pi[idx] = 2.0 * GXp[idx] * GXm[b * NN + j * N + i];
    GX[idx] = GXp[idx];
  }
}

// A[m] = Vinv - A[m] (in place) for every sampled frequency m.
__global__ void gw_shift_kernel(long long NN, long long batch, const double* __restrict__ Vinv, double* __restrict__ A) {
  const long long total = NN * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    A[idx] = Vinv[idx % NN] - A[idx];
}

// A[m] -= V (screened minus bare interaction).
__global__ void gw_sub_kernel(long long NN, long long batch, const double* __restrict__ V, double* __restrict__ A) {
  const long long total = NN * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x)
    A[idx] -= V[idx % NN];
}

// M[b][R][P] = C_SOX D[b][P][R] - GX[b][R][P] W~[b][R][P] (D may be null: GW term alone).
__global__ void gw_merge_kernel(long long N, long long batch, const double* __restrict__ D,
                                const double* __restrict__ GX, const double* __restrict__ Wt, double* __restrict__ M) {
  const long long NN = N * N, total = NN * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / NN, r = idx - b * NN, R = r / N, P = r - R * N;
    double m = -GX[idx] * Wt[idx];
    if (D) m += D[b * NN + P * N + R];
    M[idx] = m;
  }
}

struct StoreE {
  double* p;
  long long sb, sr, sc;
  __device__ __forceinline__ void operator()(long long b, long long m, long long c, double v) const {
    p[b * sb + m * sr + c * sc] = v;
  }
};

}  // namespace

// In-place inverse of `batch` SPD n x n matrices at A (no pivoting).
int gj_invert_spd(thc_ctx* ctx, double* A, long long n, long long batch) {
  if (!ctx->gw_scr)
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_scr, sizeof(double) * (size_t)std::max<long long>(batch, ctx->gw_nw + 1) *
                                                 (2 * (size_t)n + 1), "Gauss-Jordan scratch"));
  double *row = ctx->gw_scr, *col = row + batch * n, *piv = col + batch * n;
  const long long total = n * n * batch;
  for (int k = 0; k < n; ++k) {
    ProfRec rec;
    THC_TRY(prof_begin(ctx, K_SCREEN, 0.0, &rec));
    gj_pivot_kernel<<<(unsigned)batch, 256, 0, ctx->stream>>>(n, k, A, row, col, piv);
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "Gauss-Jordan pivot"));
    THC_TRY(prof_begin(ctx, K_SCREEN, 2.0 * (double)n * n * batch, &rec));
    gj_update_kernel<<<blocks_for(total), 256, 0, ctx->stream>>>(n, k, batch, A, row, col, piv);
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "Gauss-Jordan update"));
  }
  return THC_OK;
}

int gw_set_transforms(thc_ctx* ctx, int n_omega, const double* to_iw, const double* to_tau) {
  const long long N = ctx->N, NN = N * N, nt = ctx->n_tau;
  if (ctx->precision != THC_FP64)
    return fail(ctx, THC_ENOTSUP, "the screened (GW) term runs on the FP64 path only");
  if (!(ctx->terms & THC_GW)) return fail(ctx, THC_EINVAL, "context was not created with THC_GW");
  if (n_omega < 1 || !to_iw || !to_tau) return fail(ctx, THC_EINVAL, "bad bosonic transforms");
  if (ctx->gw_nw && ctx->gw_nw != n_omega)
    return fail(ctx, THC_EINVAL, "the number of bosonic frequencies cannot change");
  ctx->gw_nw = n_omega;
  if (!ctx->gw_toiw) {
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_toiw, sizeof(double) * n_omega * nt, "to_iw"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_totau, sizeof(double) * nt * n_omega, "to_tau"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_vinv, sizeof(double) * NN, "V^-1"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_pi, sizeof(double) * nt * NN, "Pi~(tau), W~(tau)"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_gx, sizeof(double) * nt * NN, "G^X(tau)"));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_w, sizeof(double) * n_omega * NN, "W(i Omega)"));
    THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->gw_vinv, ctx->V, sizeof(double) * NN, cudaMemcpyDeviceToDevice,
                                            ctx->stream), "copy V"));
    THC_TRY(gj_invert_spd(ctx, ctx->gw_vinv, N, 1));
  }
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->gw_toiw, to_iw, sizeof(double) * n_omega * nt, cudaMemcpyHostToDevice,
                                          ctx->stream), "copy to_iw"));
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->gw_totau, to_tau, sizeof(double) * nt * n_omega,
                                          cudaMemcpyHostToDevice, ctx->stream), "copy to_tau"));
  return check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "bosonic transforms sync");
}

// Pi~ and G^X of the tau points c0 .. c0 + tc - 1, from the chunk's G^X(+-tau) buffers.
int gw_store_bubble(thc_ctx* ctx, long long c0, long long tc) {
  const long long N = ctx->N, NN = N * N;
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_POLARISATION, 0.0, &rec));
  gw_bubble_kernel<<<blocks_for(NN * tc), 256, 0, ctx->stream>>>(N, tc, ctx->GXp, ctx->GXm, ctx->gw_pi + c0 * NN,
                                                                 ctx->gw_gx + c0 * NN);
  return prof_end(ctx, &rec, cudaGetLastError(), "GW bubble");
}

// W~(tau_k) for every tau point (into gw_pi) from Pi~(tau_k) (in gw_pi).
int gw_screen(thc_ctx* ctx) {
  const long long N = ctx->N, NN = N * N, nt = ctx->n_tau, nw = ctx->gw_nw;
  // Pi~(i W_m) = sum_k to_iw[m][k] Pi~(tau_k): (m, e) = sum_k A(m, k) B(k, e)
  {
    ProfRec rec;
    THC_TRY(prof_begin(ctx, K_SCREEN, 2.0 * nw * NN * nt, &rec));
    const dim3 grid((unsigned)((nw + f64::BM - 1) / f64::BM), (unsigned)((NN + f64::BN - 1) / f64::BN), 1);
    f64::gemm_kernel<true, false><<<grid, f64::NT, 0, ctx->stream>>>(
        nw, NN, nt, View{ctx->gw_toiw, 0, nt, 1}, View{ctx->gw_pi, 0, NN, 1}, StoreE{ctx->gw_w, 0, NN, 1});
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "Pi~(i Omega)"));
  }
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_SCREEN, 0.0, &rec));
  gw_shift_kernel<<<blocks_for(NN * nw), 256, 0, ctx->stream>>>(NN, nw, ctx->gw_vinv, ctx->gw_w);
  THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "V^-1 - Pi~"));
  THC_TRY(gj_invert_spd(ctx, ctx->gw_w, N, nw));  // W = (V^-1 - Pi~)^-1
  THC_TRY(prof_begin(ctx, K_SCREEN, 0.0, &rec));
  gw_sub_kernel<<<blocks_for(NN * nw), 256, 0, ctx->stream>>>(NN, nw, ctx->V, ctx->gw_w);
  THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "W - V"));
  // W~(tau_k) = sum_m to_tau[k][m] W~(i W_m)
  THC_TRY(prof_begin(ctx, K_SCREEN, 2.0 * nt * NN * nw, &rec));
  const dim3 grid((unsigned)((nt + f64::BM - 1) / f64::BM), (unsigned)((NN + f64::BN - 1) / f64::BN), 1);
  f64::gemm_kernel<true, false><<<grid, f64::NT, 0, ctx->stream>>>(
      nt, NN, nw, View{ctx->gw_totau, 0, nw, 1}, View{ctx->gw_w, 0, NN, 1}, StoreE{ctx->gw_pi, 0, NN, 1});
  return prof_end(ctx, &rec, cudaGetLastError(), "W~(tau)");
}

// M = C_SOX D^T - G^X o W~ for the tau points of a chunk (into M).
int gw_merge(thc_ctx* ctx, long long c0, long long tc, const double* D, double* M) {
  const long long N = ctx->N, NN = N * N;
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_DIRECT_W, 0.0, &rec));
  gw_merge_kernel<<<blocks_for(NN * tc), 256, 0, ctx->stream>>>(N, tc, D, ctx->gw_gx + c0 * NN, ctx->gw_pi + c0 * NN,
                                                                M);
  return prof_end(ctx, &rec, cudaGetLastError(), "GW merge");
}

}  // namespace thc

extern "C" int thc_sigma_set_bosonic(thc_ctx* ctx, int n_omega, const double* to_iw, const double* to_tau) {
  if (!ctx) return thc::fail(nullptr, THC_EINVAL, "ctx is NULL");
  try {
    return thc::gw_set_transforms(ctx, n_omega, to_iw, to_tau);
  } catch (...) {
    return thc::fail(ctx, THC_ENOMEM, "host allocation failed");
  }
}
