// Screened direct term (scGW, scGWSOX; Sec. II.C, first paragraph: the THC-GW
// scheme), its screening in FP64 on both paths.  Restricted, per spin:
//
//   Pi~(tau)   = 2 G^X(tau) o G^X(-tau)^T                   (spin-summed bubble)
//   Pi~(i W_m) = sum_k to_iw[m][k] Pi~(tau_k)                (bosonic transform)
//   W(i W_m)   = V [1 - Pi~ V]^{-1} = (V^{-1} - Pi~)^{-1}    (SPD: V SPD, Pi~ <= 0)
//   W~(tau_k)  = sum_m to_tau[k][m] (W - V)(i W_m)
//   Sigma^GW   = -X (G^X(tau) o W~(tau)) X^T
//
// Unrestricted (Sec. II.A's spin-orbitals, G block-diagonal in spin): Pi~ is the sum of
// G^X_s(tau) o G^X_s(-tau)^T over both spins, one W serves both, and Sigma^GW_s takes
// G^X_s on its outer line.
//
// W is formed as the inverse of the symmetric positive definite V^{-1} - Pi~, an
// elimination without pivoting (stable for SPD matrices), batched over the sampled
// frequencies; V^{-1} is formed the same way once per context.  Matrices up to
// 2 kGJBlock rows are eliminated one pivot at a time (Gauss-Jordan); larger ones by
// the symmetric sweep in blocks of kGJBlock pivots on the upper triangle, whose
// trailing updates (N^2 kGJBlock flops each, N^3 in all) run in the DFMA
// contraction tile.
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

// Blocked symmetric sweep (matrices of more than 2 kGJBlock rows).  Only the upper
// triangle (i <= j) of A is read or written; sym(i, j) is element (min, max).
// Step at pivots k0 .. k0 + kb - 1: CT[c][i] = sym(i, k0 + c) (n columns of kb rows)
// and P = A[k, k] copied out.
__global__ void sym_panels_kernel(long long n, long long k0, long long kb, long long batch,
                                  const double* __restrict__ A, double* __restrict__ CT, double* __restrict__ P) {
  const long long per = n * kb, total = per * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / per, e = idx - b * per, c = e / n, i = e - c * n, k = k0 + c;
    const double* a = A + b * n * n;
    const double v = i <= k ? a[i * n + k] : a[k * n + i];
    CT[idx] = v;
    if (i >= k0 && i < k0 + kb) P[b * kb * kb + c * kb + (i - k0)] = v;
  }
}

// After the trailing update, with Rp = P C^T (kb x n, P = A[k, k]^{-1}): the block row
// A[k][j] = Rp[:, j] (j > k), the block column A[i][k] = Rp[:, i]^T (i < k), and
// A[k, k] = -P.
__global__ void sym_rows_kernel(long long n, long long k0, long long kb, long long batch, const double* __restrict__ Rp,
                                const double* __restrict__ P, double* __restrict__ A) {
  const long long per = kb * n, total = per * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / per, e = idx - b * per, r = e / n, j = e - r * n;
    double* a = A + b * n * n;
    if (j < k0)
      a[j * n + k0 + r] = Rp[idx];
    else if (j < k0 + kb)
      a[(k0 + r) * n + j] = -P[b * kb * kb + r * kb + (j - k0)];
    else
      a[(k0 + r) * n + j] = Rp[idx];
  }
}

// A(b, m, c) -= v on and above the diagonal (m <= c); tiles wholly below it are skipped.
struct SymSubEpi {
  double* p;
  long long sb, sr;
  __device__ __forceinline__ void operator()(long long b, long long m, long long c, double v) const {
    if (m <= c) p[b * sb + m * sr + c] -= v;
  }
  __device__ __forceinline__ bool skip_tile(long long, long long m0, long long c_end) const { return c_end <= m0; }
};

// The sweep of every pivot leaves -A^{-1} in the upper triangle: A <- -sym(A), both
// triangles, through a 32 x 32 tile in shared memory (grid: column tile, row tile, batch).
__global__ void sym_finish_kernel(long long n, double* __restrict__ A) {
  __shared__ double t[32][33];
  const long long ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  double* a = A + (long long)blockIdx.z * n * n;
  const long long i0 = ti * 32, j0 = tj * 32;
  const int x = threadIdx.x & 31, y0 = threadIdx.x >> 5;  // 32 x 8 threads
  for (int y = y0; y < 32; y += 8) {
    const long long i = i0 + y, j = j0 + x;
    if (i < n && j < n && i <= j) t[y][x] = -a[i * n + j];
  }
  __syncthreads();
  for (int y = y0; y < 32; y += 8) {
    const long long i = i0 + y, j = j0 + x;   // upper tile, element (i, j)
    if (i < n && j < n && i <= j) a[i * n + j] = t[y][x];
    const long long il = j0 + y, jl = i0 + x;  // lower tile, element (il, jl) = (jl, il) of the upper
    if (il < n && jl < n && il > jl) a[il * n + jl] = t[x][y];
  }
}

// Pi~[k0 + b] (+)= scale GXp[b] o GXm[b]^T and GX[k0 + b] = GXp[b] for the tau points of a
// chunk (scale 2: both spins of a restricted G; 1 and accumulate: one spin after the other).
template <class T>
__global__ void gw_bubble_kernel(long long N, long long batch, const T* __restrict__ GXp, const T* __restrict__ GXm,
                                 double scale, int accumulate, double* __restrict__ Pi, double* __restrict__ GX) {
  const long long NN = N * N, total = NN * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / NN, r = idx - b * NN, i = r / N, j = r - i * N;
    const double p = scale * (double)GXp[idx] * (double)GXm[b * NN + j * N + i];
    Pi[idx] = accumulate ? Pi[idx] + p : p;
    GX[idx] = (double)GXp[idx];
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
    double m = -GX[idx] * Wt[idx];
    if (D) m += D[idx];  // D[P][R] = D[R][P]: D is mirrored to symmetric before the merge
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

constexpr long long kGJBlock = 64;  // pivots per blocked step

// One pivot at a time (matrices of up to 2 kGJBlock rows, and the diagonal blocks).
int gj_invert_unblocked(thc_ctx* ctx, double* A, long long n, long long batch, double* row, double* col,
                        double* piv) {
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

// In-place inverse of `batch` SPD n x n matrices at A (no pivoting).  Up to 2 kGJBlock
// rows: Gauss-Jordan one pivot at a time.  Above that: the symmetric sweep in blocks of
// kb pivots, which keeps the matrix symmetric at every step and so works on the upper
// triangle alone.  A step at pivots k (P = A_kk^{-1}, C = A[:, k] before the step) sets
//   A_ij -= C_i P C_j^T   (i, j outside k),   A_ik = C_i P,   A_kj = P C_j^T,   A_kk = -P;
// after every pivot has been swept the matrix holds -A^{-1}.  The trailing update,
// n^2 kb flops per step on the upper tiles, is n^3 in all (Gauss-Jordan on the full
// matrix: 2 n^3).
int gj_invert_spd(thc_ctx* ctx, double* A, long long n, long long batch) {
  const bool blocked = n > 2 * kGJBlock;
  const long long kb = std::min(n, kGJBlock);
  // scratch: row, col, piv of the one-pivot steps (of n or of kb rows), and the panels
  const long long nrow = blocked ? kb : n;
  auto elems_for = [&](long long bt) {
    return (size_t)bt * (2 * nrow + 1) + (blocked ? (size_t)bt * (2 * n * kb + kb * kb) : 0);
  };
  if (!ctx->gw_scr) {  // sized once, for the larger of this batch and the frequency count
    const size_t elems = elems_for(std::max<long long>(batch, ctx->gw_nw));
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_scr, sizeof(double) * elems, "Gauss-Jordan scratch"));
    ctx->gw_scr_elems = elems;
  }
  if (elems_for(batch) > ctx->gw_scr_elems) return fail(ctx, THC_EINVAL, "Gauss-Jordan scratch too small for this batch");
  double *row = ctx->gw_scr, *col = row + batch * nrow, *piv = col + batch * nrow;
  if (!blocked) return gj_invert_unblocked(ctx, A, n, batch, row, col, piv);
  double *CT = piv + batch, *Rp = CT + batch * n * kb, *P = Rp + batch * n * kb;
  const long long nn = n * n;
  for (long long k0 = 0; k0 < n; k0 += kGJBlock) {
    const long long b = std::min(kGJBlock, n - k0);
    ProfRec rec;
    THC_TRY(prof_begin(ctx, K_SCREEN, 0.0, &rec));
    sym_panels_kernel<<<blocks_for(n * b * batch), 256, 0, ctx->stream>>>(n, k0, b, batch, A, CT, P);
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "sweep panels"));
    THC_TRY(gj_invert_unblocked(ctx, P, b, batch, row, col, piv));  // P = A_kk^{-1}
    const dim3 gr((unsigned)((b + f64::BM - 1) / f64::BM), (unsigned)((n + f64::BN - 1) / f64::BN), (unsigned)batch);
    THC_TRY(prof_begin(ctx, K_SCREEN, 2.0 * b * n * b * batch, &rec));  // Rp = P C^T
    f64::gemm_kernel<true, false><<<gr, f64::NT, 0, ctx->stream>>>(
        b, n, b, View{P, b * b, b, 1}, View{CT, n * b, n, 1}, f64::StoreEpi{Rp, n * b, n, 1, 1.0});
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "sweep row panel"));
    const dim3 gt((unsigned)((n + f64::BM - 1) / f64::BM), (unsigned)((n + f64::BN - 1) / f64::BN), (unsigned)batch);
    THC_TRY(prof_begin(ctx, K_SCREEN, 1.0 * n * (n + f64::BN) * b * batch, &rec));  // A -= C Rp (upper tiles)
    f64::gemm_kernel<false, false><<<gt, f64::NT, 0, ctx->stream>>>(
        n, n, b, View{CT, n * b, 1, n}, View{Rp, n * b, n, 1}, SymSubEpi{A, nn, n});
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "sweep trailing update"));
    THC_TRY(prof_begin(ctx, K_SCREEN, 0.0, &rec));  // block row and column from Rp, A_kk = -P
    sym_rows_kernel<<<blocks_for(b * n * batch), 256, 0, ctx->stream>>>(n, k0, b, batch, Rp, P, A);
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "sweep block row"));
  }
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_SCREEN, 0.0, &rec));
  const dim3 gf((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)batch);
  sym_finish_kernel<<<gf, 256, 0, ctx->stream>>>(n, A);
  return prof_end(ctx, &rec, cudaGetLastError(), "sweep sign and mirror");
}

int gw_set_transforms(thc_ctx* ctx, int n_omega, const double* to_iw, const double* to_tau) {
  const long long N = ctx->N, NN = N * N, nt = ctx->n_tau;
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
    if (ctx->precision != THC_FP64)  // the merged M of a chunk before its split
      THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_m, sizeof(double) * ctx->tc * NN, "M of the screened term"));
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

// G^X of spin s for every tau point: gw_gx (restricted, or spin a) or gw_gx_b (spin b,
// allocated on the first unrestricted evaluation).
int gw_gx_of(thc_ctx* ctx, int spin, double** gx) {
  if (spin == 1 && !ctx->gw_gx_b)
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->gw_gx_b, sizeof(double) * ctx->n_tau * ctx->N * ctx->N, "G^X(tau) of spin b"));
  *gx = spin == 1 ? ctx->gw_gx_b : ctx->gw_gx;
  return THC_OK;
}

// Pi~ and G^X of the tau points c0 .. c0 + tc - 1, from the chunk's G^X(+-tau) buffers
// (FP64 path; the split path's are FP32).  nspin 1: Pi~ = 2 G^X o G^X(-)^T; nspin 2: the
// spin's own G^X o G^X(-)^T, spin b first, spin a added.
int gw_store_bubble(thc_ctx* ctx, long long c0, long long tc, int nspin, int spin) {
  const long long N = ctx->N, NN = N * N;
  double* gx = nullptr;
  THC_TRY(gw_gx_of(ctx, spin, &gx));
  const double scale = nspin == 1 ? 2.0 : 1.0;
  const int acc = nspin == 2 && spin == 0;
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_POLARISATION, 0.0, &rec));
  if (ctx->precision == THC_FP64)
    gw_bubble_kernel<double><<<blocks_for(NN * tc), 256, 0, ctx->stream>>>(N, tc, ctx->GXp, ctx->GXm, scale, acc,
                                                                         ctx->gw_pi + c0 * NN, gx + c0 * NN);
  else
    gw_bubble_kernel<float><<<blocks_for(NN * tc), 256, 0, ctx->stream>>>(N, tc, ctx->GXf, ctx->GXmf, scale, acc,
                                                                        ctx->gw_pi + c0 * NN, gx + c0 * NN);
  return prof_end(ctx, &rec, cudaGetLastError(), "GW bubble");
}

// W~(tau_k) for every tau point (into gw_pi) from Pi~(tau_k) (in gw_pi).
int gw_screen(thc_ctx* ctx) {
  const long long N = ctx->N, NN = N * N, nt = ctx->n_tau, nw = ctx->gw_nw;
  // Pi~(i W_m) = sum_k to_iw[m][k] Pi~(tau_k), as the contraction (e, m) = sum_k A(e, k) B(k, m)
  // with the N^2 elements e along the grid's first dimension (no 65535 limit there)
  {
    ProfRec rec;
    THC_TRY(prof_begin(ctx, K_SCREEN, 2.0 * nw * NN * nt, &rec));
    const dim3 grid((unsigned)((NN + f64::BM - 1) / f64::BM), (unsigned)((nw + f64::BN - 1) / f64::BN), 1);
    f64::gemm_kernel<false, true><<<grid, f64::NT, 0, ctx->stream>>>(
        NN, nw, nt, View{ctx->gw_pi, 0, 1, NN}, View{ctx->gw_toiw, 0, 1, nt}, StoreE{ctx->gw_w, 0, 1, NN});
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
  // W~(tau_k) = sum_m to_tau[k][m] W~(i W_m), as (e, k) = sum_m A(e, m) B(m, k)
  THC_TRY(prof_begin(ctx, K_SCREEN, 2.0 * nt * NN * nw, &rec));
  const dim3 grid((unsigned)((NN + f64::BM - 1) / f64::BM), (unsigned)((nt + f64::BN - 1) / f64::BN), 1);
  f64::gemm_kernel<false, true><<<grid, f64::NT, 0, ctx->stream>>>(
      NN, nt, nw, View{ctx->gw_w, 0, 1, NN}, View{ctx->gw_totau, 0, 1, nw}, StoreE{ctx->gw_pi, 0, 1, NN});
  return prof_end(ctx, &rec, cudaGetLastError(), "W~(tau)");
}

// M = C_SOX D^T - G^X_s o W~ for the tau points of a chunk (into M), G^X of spin s.
int gw_merge(thc_ctx* ctx, long long c0, long long tc, const double* D, double* M, int spin) {
  const long long N = ctx->N, NN = N * N;
  double* gx = nullptr;
  THC_TRY(gw_gx_of(ctx, spin, &gx));
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_DIRECT_W, 0.0, &rec));
  gw_merge_kernel<<<blocks_for(NN * tc), 256, 0, ctx->stream>>>(N, tc, D, gx + c0 * NN, ctx->gw_pi + c0 * NN, M);
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
