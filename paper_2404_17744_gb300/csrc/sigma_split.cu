// Split-precision (3 x BF16 on tcgen05) evaluation of the THC self-energy.
//
// Same steps and order as the FP64 path (Sec. II.C scheme plus the direct
// term), with every contraction on the tensor cores through
// tc::split_gemm_kernel: operands are BF16 hi/lo pairs, accumulation is FP32
// in TMEM, and each epilogue either re-splits its output for the next
// contraction, stores it in FP32, reduces it (the Hadamard-reduce of D_PR),
// or writes the FP64 result.  Contractions are arranged so that both
// operands are K-major:
//   Y[R][q]      = sum_u Xt[R][u] G[q][u]                      (G symmetric)
//   A^T_P[v][q]  = sum_s U[P q][s] G(-tau)[v][s]   -> stored transposed per P
//   B_P[R][v]    = sum_q Y[R][q] A^T_P[v][q]
//   D[P][R]     += sum_v (sum_w Y[P][w] U_R[v][w]) B_P[R][v]   (C never stored)
//   G^X[P][R]    = sum_q Y[P][q] Xt[R][q]
//   T[P][S]      = sum_Q V[P][Q] Pi[S][Q]                       (Pi symmetric)
//   M[R][P]      = c_x D[P][R] + c_d G^X[R][P] sum_S T[R][S] V[P][S]
//   T2t[r][R]    = sum_P M[R][P] X[r][P]        -> stored transposed
//   Sigma[t][r]  = sum_R X[t][R] T2t[r][R]
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "tc_bcd.cuh"
#include "tc_gemm.cuh"
#include "tc_soxa.cuh"
#include "thc_internal.cuh"

namespace thc {
namespace {

using bf16 = __nv_bfloat16;
using tc::Cfg;

constexpr double C_DIRECT = -2.0;
constexpr double C_SOX = +1.0;

inline long long pad8(long long x) { return (x + 7) / 8 * 8; }
// Row pitch of the split operands: a multiple of 64 elements, so that every row starts on a
// 128-byte line and a 64-deep TMA box row is one line.  Measured against pitches of 8 and 16
// elements at n = 200 (400- and 416-byte rows): the A contraction 118 and 97 us against
// 88 us per launch; the rows of unaligned pitches straddle 32-byte sectors and lines.
inline long long pad_row(long long x) { return (x + 63) / 64 * 64; }

// BF16 hi/lo pair: element (b, r, c) at hi[b * bs + r * ld + c]; lo2, when not null, is
// the third term of a constant operand (x = hi + lo + lo2 to about 24 bits).
struct Split {
  bf16* hi;
  bf16* lo;
  long long rows;
  long long ld;
  long long batch;
  long long bs;
  bf16* lo2 = nullptr;
  Split at_row(long long r0, long long nrows) const {
    return Split{hi + r0 * ld, lo + r0 * ld, nrows, ld, batch, bs, lo2 ? lo2 + r0 * ld : nullptr};
  }
  Split at_batch(long long b0, long long nb) const {
    return Split{hi + b0 * bs, lo + b0 * bs, rows, ld, nb, bs, lo2 ? lo2 + b0 * bs : nullptr};
  }
};

// ------------------------------------------------------------- tensor maps
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

int get_encoder(thc_ctx* ctx) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (g_encode) return THC_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return fail(ctx, THC_ECUDA, "cuTensorMapEncodeTiled entry point not available");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return THC_OK;
}

// 3-D map (k, row, batch) over one half of a Split, box 64 x box_rows x 1, 128-byte swizzle.
int make_map(thc_ctx* ctx, CUtensorMap* m, const bf16* base, long long K, const Split& s, int box_rows,
             int box_k = tc::BKE, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B) {
  const long long batch = std::max<long long>(1, s.batch);
  const long long bs = s.batch > 1 ? s.bs : s.rows * s.ld;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)s.rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(s.ld * 2), (cuuint64_t)(bs * 2)};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (s.ld * 2) % 16 || (bs * 2) % 16)
    return fail(ctx, THC_EINVAL, "tensor map operand not 16-byte aligned");
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, THC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return THC_OK;
}

// 3-D map with explicit extents (elements), byte strides of dims 1 and 2, and box; 128-byte
// swizzle (operand loads) or none (the store boxes of the A contraction).
int make_map_3d(thc_ctx* ctx, CUtensorMap* m, const bf16* base, const long long dims_in[3], const long long strides_in[2],
                const int box_in[3], CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_128B) {
  cuuint64_t dims[3] = {(cuuint64_t)dims_in[0], (cuuint64_t)dims_in[1], (cuuint64_t)dims_in[2]};
  cuuint64_t strides[2] = {(cuuint64_t)strides_in[0], (cuuint64_t)strides_in[1]};
  cuuint32_t box[3] = {(cuuint32_t)box_in[0], (cuuint32_t)box_in[1], (cuuint32_t)box_in[2]};
  cuuint32_t es[3] = {1, 1, 1};
  if ((reinterpret_cast<uintptr_t>(base) & 15) || strides[0] % 16 || strides[1] % 16)
    return fail(ctx, THC_EINVAL, "tensor map operand not 16-byte aligned");
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, THC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return THC_OK;
}

// ------------------------------------------------------------ epilogues
// Each functor is run by one warp on a 32 x 32 chunk of the output tile:
// t(r, j) = C[row0 + r][col0 + j]; rows >= M and columns >= N are skipped.
using Tile = tc::TileRef;

__device__ __forceinline__ void split_store(bf16* hi, bf16* lo, long long o, float v) {
  const bf16 h = __float2bfloat16_rn(v);
  hi[o] = h;
  lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// hi, lo and, when lo2 is set, the third term of v (the FP32 value exactly, 24 bits)
__device__ __forceinline__ void split_store3(bf16* hi, bf16* lo, bf16* lo2, long long o, float v) {
  const bf16 h = __float2bfloat16_rn(v);
  const float r = v - __bfloat162float(h);
  const bf16 l = __float2bfloat16_rn(r);
  hi[o] = h;
  lo[o] = l;
  if (lo2) lo2[o] = __float2bfloat16_rn(r - __bfloat162float(l));
}

// dst(b, row, col) = scale * C, split; row-major, or transposed dst(b, col, row).
// With lo2 set the third term is stored too.
template <bool TRANSPOSED>
struct EpiSplit {
  bf16 *hi, *lo;
  long long ld, bs;
  float scale;
  bf16* lo2 = nullptr;
  __device__ void operator()(int b, int row0, int col0, Tile t, int lane, int M, int N) const {
    if (TRANSPOSED) {  // lanes along rows: dst(b, col, row) is contiguous in row
      const int row = row0 + lane;
      if (row >= M) return;
#pragma unroll 4
      for (int j = 0; j < 32; ++j)
        if (col0 + j < N)
          split_store3(hi, lo, lo2, (long long)b * bs + (long long)(col0 + j) * ld + row, scale * t(lane, j));
    } else {           // lanes along columns
      const int col = col0 + lane;
      if (col >= N) return;
#pragma unroll 4
      for (int r = 0; r < 32; ++r)
        if (row0 + r < M)
          split_store3(hi, lo, lo2, (long long)b * bs + (long long)(row0 + r) * ld + col, scale * t(r, lane));
    }
  }
};

// FP32 store: dst[b * bs + row * ld + col] (lanes along columns).
struct EpiF32 {
  float* dst;
  long long ld, bs;
  __device__ void operator()(int b, int row0, int col0, Tile t, int lane, int M, int N) const {
    const int col = col0 + lane;
    if (col >= N) return;
    float* d = dst + (long long)b * bs + col;
#pragma unroll 4
    for (int r = 0; r < 32; ++r)
      if (row0 + r < M) d[(long long)(row0 + r) * ld] = t(r, lane);
  }
};

// FP64 store: dst[b * bs + row * ld + col] (lanes along columns).
struct EpiF64 {
  double* dst;
  long long ld, bs;
  __device__ void operator()(int b, int row0, int col0, Tile t, int lane, int M, int N) const {
    const int col = col0 + lane;
    if (col >= N) return;
    double* d = dst + (long long)b * bs + col;
#pragma unroll 4
    for (int r = 0; r < 32; ++r)
      if (row0 + r < M) d[(long long)(row0 + r) * ld] = (double)t(r, lane);
  }
};

// Merge epilogue of W = T V: M[b][R][P] = c_x D[b][P][R] + cd G^X[b][R][P] W, split (lanes along P);
// cd = C_DIRECT for a restricted G, -1 per spin of an unrestricted one (Pi summed over both spins).
struct EpiMerge {
  bf16 *hi, *lo;
  long long ld;
  const double* D;  // may be null
  const float* GX;
  int N;
  double cd;
  bf16* lo2 = nullptr;  // third term of M, when set
  __device__ void operator()(int b, int row0, int col0, Tile t, int lane, int M, int Ncols) const {
    const int P = col0 + lane;
    if (P >= Ncols) return;
    const long long NN = (long long)N * N;
    // 16 rows at a time: all their G^X and D loads are issued before the first is used
    for (int r0 = 0; r0 < 32; r0 += 16) {
      float gx[16];
      double dv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int R = row0 + r0 + i;
        const long long o = b * NN + (long long)R * N + P;
        gx[i] = R < M ? GX[o] : 0.f;
        dv[i] = (D && R < M) ? D[o] : 0.0;  // D is symmetric (mirrored): D[P][R] = D[R][P]
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int R = row0 + r0 + i;
        if (R >= M) return;
        const double m = cd * (double)gx[i] * (double)t(r0 + i, lane) + C_SOX * dv[i];
        split_store3(hi, lo, lo2, (long long)b * N * ld + (long long)R * ld + P, (float)m);
      }
    }
  }
};

// U build: row = P, col = (q - q0) n + s  ->  U[(P n + q) ld + s], split (lanes along s).
struct EpiU {
  bf16 *hi, *lo;
  int n, q0;
  long long ld;
  __device__ void operator()(int, int row0, int col0, Tile t, int lane, int M, int Ncols) const {
    const int c = col0 + lane;
    if (c >= Ncols) return;
    const int q = q0 + c / n, s = c - (c / n) * n;
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      const int P = row0 + r;
      if (P >= M) break;
      split_store(hi, lo, ((long long)P * n + q) * ld + s, t(r, lane));
    }
  }
};

// --------------------------------------------------------- split kernels
// dst(b, r, c) = split(scale * src[b sb + r sr + c sc]) for c < cols; 0 on the padding cols..ld.
// With lo2 non-null the residual x - hi - lo is kept as a third term.
__global__ void split_f64_kernel(const double* __restrict__ src, long long sb, long long sr, long long sc,
                                 double scale, bf16* __restrict__ hi, bf16* __restrict__ lo, bf16* __restrict__ lo2,
                                 long long rows, long long cols, long long ld, long long batch, long long dbs) {
  const long long per = rows * ld, total = per * batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / per, rem = i - b * per, r = rem / ld, c = rem - r * ld;
    const long long o = b * dbs + r * ld + c;
    if (c < cols) {
      const double x = scale * src[b * sb + r * sr + c * sc];
      const bf16 h = __float2bfloat16_rn((float)x);
      const double r1 = x - (double)__bfloat162float(h);
      const bf16 l = __float2bfloat16_rn((float)r1);
      hi[o] = h;
      lo[o] = l;
      if (lo2) lo2[o] = __float2bfloat16_rn((float)(r1 - (double)__bfloat162float(l)));
    } else {
      hi[o] = __float2bfloat16_rn(0.f);
      lo[o] = __float2bfloat16_rn(0.f);
      if (lo2) lo2[o] = __float2bfloat16_rn(0.f);
    }
  }
}

// Khatri-Rao block of the U build: KR[(q - q0) n + s][Q] = X[q][Q] X[s][Q], split, ld >= N.
__global__ void kr_split_kernel(const double* __restrict__ X, int n, int N, int q0, int qb, bf16* __restrict__ hi,
                                bf16* __restrict__ lo, long long ld) {
  const long long total = (long long)qb * n * ld;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / ld, Q = i - r * ld;
    const int q = q0 + (int)(r / n), s = (int)(r % n);
    if (Q < N) {
      const double x = X[(long long)q * N + Q] * X[(long long)s * N + Q];
      const bf16 h = __float2bfloat16_rn((float)x);
      hi[i] = h;
      lo[i] = __float2bfloat16_rn((float)(x - (double)__bfloat162float(h)));
    } else {
      hi[i] = __float2bfloat16_rn(0.f);
      lo[i] = __float2bfloat16_rn(0.f);
    }
  }
}

// Pi[b][Q][S] = G^X[b][Q][S] G^X(-)[b][S][Q] (+ add[b][Q][S], the FP32 polarisation of the
// other spin, when add is set), split; with keep set, the FP32 value is stored there instead.
__global__ void polarisation_split_kernel(long long N, long long batch, const float* __restrict__ GX,
                                          const float* __restrict__ GXm, const float* __restrict__ add,
                                          float* __restrict__ keep, bf16* __restrict__ hi, bf16* __restrict__ lo,
                                          bf16* __restrict__ lo2, long long ld) {
  const long long per = N * ld, total = per * batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / per, rem = i - b * per, q = rem / ld, s = rem - q * ld;
    float v = 0.f;
    if (s < N) {
      const long long o = b * N * N + q * N + s;
      v = GX[o] * GXm[b * N * N + s * N + q];
      if (add) v += add[o];
      if (keep) {
        keep[o] = v;
        continue;
      }
    }
    if (keep) continue;
    const bf16 h = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(h);
    const bf16 l = __float2bfloat16_rn(r);
    hi[i] = h;
    lo[i] = l;
    if (lo2) lo2[i] = __float2bfloat16_rn(r - __bfloat162float(l));
  }
}

inline int blocks_for(long long total) { return (int)std::min<long long>((total + 255) / 256, 152LL * 32); }

int launch_split_f64(thc_ctx* ctx, const double* src, long long sb, long long sr, long long sc, double scale,
                     const Split& d, long long cols, const char* what) {
  const long long total = d.rows * d.ld * std::max<long long>(1, d.batch);
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_SPLIT, 0.0, &rec));
  split_f64_kernel<<<blocks_for(total), 256, 0, ctx->stream>>>(src, sb, sr, sc, scale, d.hi, d.lo, d.lo2, d.rows, cols,
                                                               d.ld, std::max<long long>(1, d.batch), d.bs);
  return prof_end(ctx, &rec, cudaGetLastError(), what);
}

// ----------------------------------------------------------- GEMM launch
// C[b](M x N) = A[b](M x K) B[b](N x K)^T in split precision; epi consumes C.
// AT = 3 multiplies the third term of A as well (A.lo2 must be set).
template <int BN, bool MULTI, class Epi, int AT = 2, int BT = 2>
int launch_split_gemm(thc_ctx* ctx, int kclass, const Split& A, bool a_batched, const Split& B, bool b_batched,
                      long long M, long long N, long long K, long long batch, const Epi& epi, const char* what) {
  if (M <= 0 || N <= 0 || batch <= 0) return THC_OK;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX || batch > INT32_MAX)
    return fail(ctx, THC_EINVAL, std::string(what) + ": contraction too large");
  if ((AT == 3 && !A.lo2) || (BT == 3 && !B.lo2))
    return fail(ctx, THC_EINVAL, std::string(what) + ": third operand term missing");
  CUtensorMap ah, al, al2, bh, bl, bl2;
  THC_TRY(make_map(ctx, &ah, A.hi, K, A, tc::BM));
  THC_TRY(make_map(ctx, &al, A.lo, K, A, tc::BM));
  THC_TRY(make_map(ctx, &al2, AT == 3 ? A.lo2 : A.lo, K, A, tc::BM));
  THC_TRY(make_map(ctx, &bh, B.hi, K, B, BN));
  THC_TRY(make_map(ctx, &bl, B.lo, K, B, BN));
  THC_TRY(make_map(ctx, &bl2, BT == 3 ? B.lo2 : B.lo, K, B, BN));
  auto kern = tc::split_gemm_kernel<BN, MULTI, AT, Epi, BT>;
  using CfgE = tc::Cfg<BN, AT, BT>;
  int sms = 0;  // the kernel's shared-memory attribute is set once per device with it
  THC_TRY(per_device(reinterpret_cast<const void*>(kern), &sms, [&](int dev, int* v) {
    THC_TRY(check_cuda(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CfgE::SMEM),
                       "split gemm smem attribute"));
    return check_cuda(ctx, cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev), "SM count");
  }));
  const long long tiles = ((M + tc::BM - 1) / tc::BM) * ((N + BN - 1) / BN) * batch;
  const dim3 grid((unsigned)std::min<long long>(tiles, sms), 1, 1);  // persistent: one CTA per SM at most
  ProfRec rec;
  THC_TRY(prof_begin(ctx, kclass, 2.0 * M * N * K * batch, &rec));
  kern<<<grid, tc::NTHREADS, CfgE::SMEM, ctx->stream>>>(ah, al, al2, bh, bl, bl2, (int)M, (int)N, (int)K, (int)batch,
                                                            tc::Operands{a_batched ? 1 : 0, b_batched ? 1 : 0}, epi,
                                                            ctx->d_err);
  return prof_end(ctx, &rec, cudaGetLastError(), what);
}

// ------------------------------------------------------------- autotuner
// The table holds, per contraction shape, the tile width (BN = 128 or 256 output
// columns) of a single-chunk contraction, and per block of the fused B C/D kernel its
// cluster shape (1 x 1, 1 x 2 or 2 x 2 CTAs).  A shape not in the table gets the width
// with the fewest padded columns (ties: 256), or 1 x 2 clusters; a context in tuning
// mode times every choice on its first encounter of a shape (CUDA events on its
// stream) and records the fastest.  Timing runs the contraction once per choice, so
// the outputs of a tuning evaluation are discarded.
struct ShapeKey {
  int kclass;
  long long M, N, K, batch;
  bool operator<(const ShapeKey& o) const {
    if (kclass != o.kclass) return kclass < o.kclass;
    if (M != o.M) return M < o.M;
    if (N != o.N) return N < o.N;
    if (K != o.K) return K < o.K;
    return batch < o.batch;
  }
};
std::map<ShapeKey, int> g_tile_table;
std::mutex g_tile_mu;

// K up to kSingleChunkK accumulates inside TMEM (single-chunk mode); longer K
// is promoted to FP32 registers every stage, with BN = 128 so the register
// accumulator does not spill.
constexpr long long kSingleChunkK = 256;

template <class Epi>
int gemm(thc_ctx* ctx, int kclass, const Split& A, bool ab, const Split& B, bool bb, long long M, long long N,
         long long K, long long batch, const Epi& epi, const char* what) {
  if (A.lo2 && B.lo2)  // three-term X or V against a three-term data operand: six products
    return launch_split_gemm<128, true, Epi, 3, 3>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
  if (A.lo2)  // three-term A operand (X or V): promoted, BN = 128 (five operand tiles per stage)
    return launch_split_gemm<128, true, Epi, 3>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
  if (K > kSingleChunkK) return launch_split_gemm<128, true>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
  const ShapeKey key{kclass, M, N, K, batch};
  int bn = 0;
  {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    auto it = g_tile_table.find(key);
    if (it != g_tile_table.end()) bn = it->second;
  }
  if (!bn && ctx->tuning && !ctx->prof_on) {
    cudaEvent_t e[3];
    for (auto& x : e) THC_TRY(check_cuda(ctx, cudaEventCreate(&x), "tuning event"));
    float t128 = 0.f, t256 = 0.f;
    int rc = check_cuda(ctx, cudaEventRecord(e[0], ctx->stream), "tuning event");
    if (rc == THC_OK) rc = launch_split_gemm<128, false>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
    if (rc == THC_OK) rc = check_cuda(ctx, cudaEventRecord(e[1], ctx->stream), "tuning event");
    if (rc == THC_OK) rc = launch_split_gemm<256, false>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
    if (rc == THC_OK) rc = check_cuda(ctx, cudaEventRecord(e[2], ctx->stream), "tuning event");
    if (rc == THC_OK) rc = check_cuda(ctx, cudaEventSynchronize(e[2]), "tuning sync");
    if (rc == THC_OK) rc = check_cuda(ctx, cudaEventElapsedTime(&t128, e[0], e[1]), "tuning time");
    if (rc == THC_OK) rc = check_cuda(ctx, cudaEventElapsedTime(&t256, e[1], e[2]), "tuning time");
    for (auto& x : e) cudaEventDestroy(x);
    THC_TRY(rc);
    std::lock_guard<std::mutex> lock(g_tile_mu);
    g_tile_table[key] = (t256 <= t128) ? 256 : 128;
    return THC_OK;
  }
  if (!bn) {
    const long long w128 = (N + 127) / 128 * 128, w256 = (N + 255) / 256 * 256;
    bn = (w256 <= w128) ? 256 : 128;
  }
  if (bn == 256) return launch_split_gemm<256, false>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
  return launch_split_gemm<128, false>(ctx, kclass, A, ab, B, bb, M, N, K, batch, epi, what);
}

Split split_of(bf16* hi, bf16* lo, long long rows, long long ld, long long batch = 1) {
  return Split{hi, lo, rows, ld, batch, rows * ld};
}
Split split3_of(bf16* hi, bf16* lo, bf16* lo2, long long rows, long long ld, long long batch = 1) {
  return Split{hi, lo, rows, ld, batch, rows * ld, lo2};
}

// Fused B and C/D of one tau point and P block (tc::sox_bcd_kernel):
//   D[P0 + P][R] += sum_v (sum_w Y[P0 + P][w] U[R][v][w]) (sum_q A^T[P][v][q] Y[R][q])
// for P0 + P <= R only (D is symmetric; the caller mirrors it).
// Y: N x ldn rows of the tau point; U: [R][v][w]; At: [P][v][q] with Pc blocks of P.
// CP x CR is the cluster shape (operand slices multicast within it).
template <int CP, int CR>
int launch_bcd_shape(thc_ctx* ctx, const Split& Y, const Split& U, const Split& At, long long P0, long long Pc,
                     double* D) {
  constexpr int CS = CP * CR;
  const long long n = ctx->n, N = ctx->N, ldn = ctx->ldn;
  tc::BcdMaps mh, ml;
  const long long udims[3] = {n, n, N}, adims[3] = {n, n, Pc};
  const long long strides[2] = {ldn * 2, n * ldn * 2};
  const int ubox[3] = {tc::BKE, 1, tc::BM / CP}, abox[3] = {tc::BKE, 1, tc::BM / CR};
  // a last K block of at most 32 columns (after at least one full one) is loaded for both
  // products into one stage, with boxes of 16 or 32 columns (32- or 64-byte swizzle)
  const long long rem = n % tc::BKE;
  const int tail = (n > tc::BKE && rem > 0) ? (rem <= 16 ? 16 : rem <= 32 ? 32 : 0) : 0;
  const CUtensorMapSwizzle tsw = tail == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B;
  const int utbox[3] = {tail, 1, tc::BM / CP}, atbox[3] = {tail, 1, tc::BM / CR};
  for (int h = 0; h < 2; ++h) {
    tc::BcdMaps& m = h ? ml : mh;
    const bf16* y = h ? Y.lo : Y.hi;
    THC_TRY(make_map(ctx, &m.yp, y, n, Y, tc::BM / CR));
    THC_TRY(make_map(ctx, &m.yr, y, n, Y, tc::BM / CP));
    THC_TRY(make_map_3d(ctx, &m.u, h ? U.lo : U.hi, udims, strides, ubox));
    THC_TRY(make_map_3d(ctx, &m.at, h ? At.lo : At.hi, adims, strides, abox));
    if (tail) {
      THC_TRY(make_map(ctx, &m.ypt, y, n, Y, tc::BM / CR, tail, tsw));
      THC_TRY(make_map(ctx, &m.yrt, y, n, Y, tc::BM / CP, tail, tsw));
      THC_TRY(make_map_3d(ctx, &m.ut, h ? U.lo : U.hi, udims, strides, utbox, tsw));
      THC_TRY(make_map_3d(ctx, &m.att, h ? At.lo : At.hi, adims, strides, atbox, tsw));
    } else {
      m.ypt = m.yp;
      m.yrt = m.yr;
      m.ut = m.u;
      m.att = m.at;
    }
  }
  auto kern = tc::sox_bcd_kernel<CP, CR>;
  int max_clusters = 0;  // resident clusters of this shape on the current device
  THC_TRY(per_device(reinterpret_cast<const void*>(kern), &max_clusters, [&](int dev, int* out) {
    THC_TRY(check_cuda(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::BcdCfg::SMEM),
                       "fused B C/D smem attribute"));
    int sms = 0;
    THC_TRY(check_cuda(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count"));
    int mc = sms / CS;
    if (CS > 1) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CS;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(mc * CS), 1, 1);
      cfg.blockDim = dim3(tc::NTHREADS, 1, 1);
      cfg.dynamicSmemBytes = tc::BcdCfg::SMEM;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int q = 0;
      THC_TRY(check_cuda(ctx, cudaOccupancyMaxActiveClusters(&q, kern, &cfg), "fused B C/D cluster occupancy"));
      mc = std::min(mc, q);
    }
    if (mc < 1) return fail(ctx, THC_ENOTSUP, "fused B C/D: no cluster of this shape fits on the device");
    *out = mc;
    return THC_OK;
  }));
  // v chunks per cluster tile: fewest v steps on the busiest SM, one more per unit for its flush
  // cluster tiles that reach R >= P (the kernel's enumeration) and the (P, R) pairs they cover
  const long long tm = (Pc + tc::BM - 1) / tc::BM, tn = (N + tc::BM - 1) / tc::BM;
  const long long tm2 = (tm + CP - 1) / CP, tn2 = (tn + CR - 1) / CR, hp = CP * tc::BM, wr = CR * tc::BM;
  long long ctiles = 0;
  double pairs = 0.0;
  for (long long i = 0; i < tm2; ++i) {
    const long long c0 = (P0 + i * hp) / wr, rows = std::min(Pc, (i + 1) * hp) - i * hp;
    if (c0 >= tn2) continue;
    ctiles += tn2 - c0;
    pairs += (double)rows * (double)(N - c0 * wr);
  }
  int nvc = 1;
  long long best = -1;
  for (long long c = 1; c <= std::min<long long>(n, 64); ++c) {
    const long long waves = (ctiles * c + max_clusters - 1) / max_clusters, cost = waves * ((n + c - 1) / c + 1);
    if (best < 0 || cost < best) {
      best = cost;
      nvc = (int)c;
    }
  }
  const long long clusters = std::min<long long>(ctiles * nvc, max_clusters);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(clusters * CS), 1, 1);
  cfg.blockDim = dim3(tc::NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = tc::BcdCfg::SMEM;
  cfg.stream = ctx->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_SOX_BCD, 2.0 * 2.0 * pairs * n * n, &rec));  // the tiles computed
  const cudaError_t e =
      cudaLaunchKernelEx(&cfg, kern, mh, ml, tc::BcdArgs{(int)Pc, (int)P0, (int)N, (int)n, nvc, tail, D}, ctx->d_err);
  return prof_end(ctx, &rec, e == cudaSuccess ? cudaGetLastError() : e, "B C/D");
}

// SOX contraction A of one tau point and P block (tc::sox_a_kernel):
//   A^T[P][v][q] = sum_s U[P0 + P][q][s] G(-tau)[v][s],  split, P < Pc
// U: the block's rows (P0 + P) n + q (K = s); G: rows v of G(-tau) (its sign included).
int launch_sox_a(thc_ctx* ctx, const Split& U, const Split& G, const Split& At, long long Pc) {
  if (Pc <= 0) return THC_OK;
  using C = tc::SoxACfg;
  const long long n = ctx->n, ldn = ctx->ldn;
  if (Pc * n > INT32_MAX) return fail(ctx, THC_EINVAL, "A: block too large");
  const int brows = (int)std::min<long long>(C::BV, (n + 15) / 16 * 16);
  tc::SoxAMaps m;
  THC_TRY(make_map(ctx, &m.uh, U.hi, n, U, tc::BM));
  THC_TRY(make_map(ctx, &m.ul, U.lo, n, U, tc::BM));
  THC_TRY(make_map(ctx, &m.gh, G.hi, n, G, brows));
  THC_TRY(make_map(ctx, &m.gl, G.lo, n, G, brows));
  const long long rem = n % tc::BKE;
  const int tail = (rem > 0 && rem <= 16) ? 16 : (rem > 16 && rem <= 32) ? 32 : 0;
  if (tail) {  // narrow boxes of the last K block (32- or 64-byte swizzle)
    const CUtensorMapSwizzle sw = tail == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B;
    THC_TRY(make_map(ctx, &m.uth, U.hi, n, U, tc::BM, tail, sw));
    THC_TRY(make_map(ctx, &m.utl, U.lo, n, U, tc::BM, tail, sw));
    THC_TRY(make_map(ctx, &m.gth, G.hi, n, G, brows, tail, sw));
    THC_TRY(make_map(ctx, &m.gtl, G.lo, n, G, brows, tail, sw));
  } else {
    m.uth = m.uh;
    m.utl = m.ul;
    m.gth = m.gh;
    m.gtl = m.gl;
  }
  const long long dims[3] = {n, n, Pc}, strides[2] = {ldn * 2, n * ldn * 2};
  const int box[3] = {tc::BM, C::CHUNK, 1};
  THC_TRY(make_map_3d(ctx, &m.ath, At.hi, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE));
  THC_TRY(make_map_3d(ctx, &m.atl, At.lo, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE));
  tc::SoxAArgs args;
  args.Pc = (int)Pc;
  args.n = (int)n;
  args.nh = (int)((n + tc::BM - 1) / tc::BM);
  args.nvt = (int)((n + C::BV - 1) / C::BV);
  args.brows = brows;
  args.tx = (uint32_t)(2 * (tc::BM + brows) * tc::BKE * 2);
  args.tail = tail;
  int sms = 0;
  THC_TRY(per_device(reinterpret_cast<const void*>(tc::sox_a_kernel), &sms, [&](int dev, int* v) {
    THC_TRY(check_cuda(ctx, cudaFuncSetAttribute(tc::sox_a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM),
                       "A smem attribute"));
    return check_cuda(ctx, cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev), "SM count");
  }));
  const long long items = Pc * args.nh * args.nvt;
  const dim3 grid((unsigned)std::min<long long>(items, sms), 1, 1);
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_SOX_A, 2.0 * Pc * n * n * n, &rec));
  tc::sox_a_kernel<<<grid, tc::NTHREADS, C::SMEM, ctx->stream>>>(m, args, ctx->d_err);
  return prof_end(ctx, &rec, cudaGetLastError(), "A");
}

// Cluster shapes of the fused B C/D kernel the autotuner chooses from, coded 10 CP + CR.
// Without a table entry: pairs of CTAs along R sharing the P-side operands, measured on
// GB300 at 200 and 500 AOs against a single CTA (-31% and -20% time) and a 2 x 2 cluster
// (-9% and -2%).
constexpr int kBcdShapes[3] = {12, 11, 22};

int launch_bcd_code(thc_ctx* ctx, int code, const Split& Y, const Split& U, const Split& At, long long P0,
                    long long Pc, double* D) {
  switch (code) {
    case 11: return launch_bcd_shape<1, 1>(ctx, Y, U, At, P0, Pc, D);
    case 22: return launch_bcd_shape<2, 2>(ctx, Y, U, At, P0, Pc, D);
    default: return launch_bcd_shape<1, 2>(ctx, Y, U, At, P0, Pc, D);
  }
}

int launch_bcd(thc_ctx* ctx, const Split& Y, const Split& U, const Split& At, long long P0, long long Pc,
               double* D) {
  if (Pc <= 0) return THC_OK;
  const ShapeKey key{K_SOX_BCD, Pc, ctx->N, ctx->n, P0};
  int code = 0;
  {
    std::lock_guard<std::mutex> lock(g_tile_mu);
    auto it = g_tile_table.find(key);
    if (it != g_tile_table.end()) code = it->second;
  }
  if (!code && ctx->tuning && !ctx->prof_on) {
    // time every shape once on this block (each adds into D: a tuning evaluation's
    // output is discarded) and record the fastest
    cudaEvent_t e[4];
    for (auto& x : e) THC_TRY(check_cuda(ctx, cudaEventCreate(&x), "tuning event"));
    float best = 0.f;
    int rc = check_cuda(ctx, cudaEventRecord(e[0], ctx->stream), "tuning event");
    for (int i = 0; i < 3 && rc == THC_OK; ++i) {
      rc = launch_bcd_code(ctx, kBcdShapes[i], Y, U, At, P0, Pc, D);
      if (rc == THC_OK) rc = check_cuda(ctx, cudaEventRecord(e[i + 1], ctx->stream), "tuning event");
    }
    if (rc == THC_OK) rc = check_cuda(ctx, cudaEventSynchronize(e[3]), "tuning sync");
    for (int i = 0; i < 3 && rc == THC_OK; ++i) {
      float ms = 0.f;
      rc = check_cuda(ctx, cudaEventElapsedTime(&ms, e[i], e[i + 1]), "tuning time");
      if (rc == THC_OK && (i == 0 || ms < best)) {
        best = ms;
        code = kBcdShapes[i];
      }
    }
    for (auto& x : e) cudaEventDestroy(x);
    THC_TRY(rc);
    std::lock_guard<std::mutex> lock(g_tile_mu);
    g_tile_table[key] = code;
    return THC_OK;
  }
  return launch_bcd_code(ctx, code ? code : kBcdShapes[0], Y, U, At, P0, Pc, D);
}

}  // namespace

// ------------------------------------------------------------------ init
int split_init(thc_ctx* ctx, size_t budget) {
  THC_TRY(get_encoder(ctx));
  const long long n = ctx->n, N = ctx->N;
  const long long ldn = pad_row(n), ldN = pad_row(N);
  ctx->ldn = (int)ldn;
  ctx->ldN = (int)ldN;
  const size_t h = sizeof(bf16);
  auto pair = [&](bf16** hi, bf16** lo, size_t elems, const char* what) -> int {
    THC_TRY(ctx_alloc(ctx, (void**)hi, h * elems, what));
    return ctx_alloc(ctx, (void**)lo, h * elems, what);
  };
  THC_TRY(pair(&ctx->Xt_h, &ctx->Xt_l, N * ldn, "Xt"));
  THC_TRY(pair(&ctx->Xs_h, &ctx->Xs_l, n * ldN, "Xs"));
  THC_TRY(pair(&ctx->Vs_h, &ctx->Vs_l, N * ldN, "Vs"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->Xt_l2, h * N * ldn, "Xt third term"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->Xs_l2, h * n * ldN, "Xs third term"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->Vs_l2, h * N * ldN, "Vs third term"));
  // blocking: per tau point and per P of the SOX block
  const size_t per_t = h * 3 * (2 * n * ldn + 2 * N * ldn + 3 * N * ldN + n * ldN) + 4 * 2 * N * N + 8 * N * N;
  const size_t per_p = h * 2 * n * ldn;
  const bool sox = ctx->terms & THC_SOX;
  if (sox) THC_TRY(pair(&ctx->Us_h, &ctx->Us_l, (size_t)N * n * ldn, "U"));
  size_t pb = std::max<size_t>(1, (budget / 2) / per_p);
  pb = std::min<size_t>(pb, (size_t)std::min<long long>(N, 65535));
  const size_t rest = budget > pb * per_p ? budget - pb * per_p : 0;
  size_t tc = std::max<size_t>(1, rest / per_t);
  tc = std::min<size_t>(tc, (size_t)std::min(ctx->n_tau, 65535));
  ctx->Pb = (int)pb;
  ctx->tc = (int)tc;
  auto triple = [&](bf16** hi, bf16** lo, bf16** lo2, size_t elems, const char* what) -> int {
    THC_TRY(pair(hi, lo, elems, what));
    return ctx_alloc(ctx, (void**)lo2, h * elems, what);
  };
  THC_TRY(triple(&ctx->Gs_h, &ctx->Gs_l, &ctx->Gs_l2, tc * n * ldn, "G split"));
  THC_TRY(triple(&ctx->Gms_h, &ctx->Gms_l, &ctx->Gms_l2, tc * n * ldn, "G(-tau) split"));
  THC_TRY(triple(&ctx->Ys_h, &ctx->Ys_l, &ctx->Ys_l2, tc * N * ldn, "Y split"));
  THC_TRY(triple(&ctx->Yms_h, &ctx->Yms_l, &ctx->Yms_l2, tc * N * ldn, "Ym split"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->GXf, 4 * tc * N * N, "G^X"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->GXmf, 4 * tc * N * N, "G^X(-)"));
  THC_TRY(triple(&ctx->Pis_h, &ctx->Pis_l, &ctx->Pis_l2, tc * N * ldN, "Pi split"));
  THC_TRY(triple(&ctx->Ts_h, &ctx->Ts_l, &ctx->Ts_l2, tc * N * ldN, "V Pi split"));
  THC_TRY(triple(&ctx->Ms_h, &ctx->Ms_l, &ctx->Ms_l2, tc * N * ldN, "M split"));
  THC_TRY(triple(&ctx->T2s_h, &ctx->T2s_l, &ctx->T2s_l2, tc * n * ldN, "T2 split"));
  THC_TRY(ctx_alloc(ctx, (void**)&ctx->Dd, 8 * tc * N * N, "D"));
  if (sox) {
    THC_TRY(pair(&ctx->Ats_h, &ctx->Ats_l, pb * n * ldn, "A^T blocks"));
  }
  // constant operands
  THC_TRY(launch_split_f64(ctx, ctx->X, 0, 1, N, 1.0, split3_of(ctx->Xt_h, ctx->Xt_l, ctx->Xt_l2, N, ldn), n,
                           "split X^T"));
  THC_TRY(launch_split_f64(ctx, ctx->X, 0, N, 1, 1.0, split3_of(ctx->Xs_h, ctx->Xs_l, ctx->Xs_l2, n, ldN), N,
                           "split X"));
  THC_TRY(launch_split_f64(ctx, ctx->V, 0, N, 1, 1.0, split3_of(ctx->Vs_h, ctx->Vs_l, ctx->Vs_l2, N, ldN), N,
                           "split V"));
  if (!sox) return THC_OK;
  // U_Pqs = sum_Q V_PQ X_qQ X_sQ over blocks of q with the Khatri-Rao block materialised
  long long qb = std::max<long long>(1, std::min<long long>(n, (long long)(budget / 2 / (h * 2 * n * ldN))));
  bf16 *kh = nullptr, *kl = nullptr;
  THC_TRY(pair(&kh, &kl, (size_t)qb * n * ldN, "Khatri-Rao block"));
  for (long long q0 = 0; q0 < n; q0 += qb) {
    const long long nq = std::min(qb, n - q0);
    ProfRec rec;
    THC_TRY(prof_begin(ctx, K_SPLIT, 0.0, &rec));
    kr_split_kernel<<<blocks_for(nq * n * ldN), 256, 0, ctx->stream>>>(ctx->X, (int)n, (int)N, (int)q0, (int)nq, kh,
                                                                        kl, ldN);
    THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "Khatri-Rao block"));
    THC_TRY(gemm(ctx, K_UBUILD, split3_of(ctx->Vs_h, ctx->Vs_l, ctx->Vs_l2, N, ldN), false, split_of(kh, kl, nq * n, ldN), false,
                 N, nq * n, N, 1, EpiU{ctx->Us_h, ctx->Us_l, (int)n, (int)q0, ldn}, "U build"));
  }
  // the Khatri-Rao block is released at init's end; keep the stream ordered first
  THC_TRY(check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "U build sync"));
  for (auto it = ctx->owned.begin(); it != ctx->owned.end();) {
    if (*it == kh || *it == kl) {
      cudaFree(*it);
      it = ctx->owned.erase(it);
    } else {
      ++it;
    }
  }
  return status_check(ctx);
}

// ------------------------------------------------------------------ eval
namespace {

// Split G(tau_k) and G(-tau_k) = -G(beta - tau_k) of one spin and chunk, then Y = X^T G(tau),
// and with the direct term Ym = X^T G(-tau) and G^X(+-tau) (G^X(-tau) only when need_minus).
int split_project(thc_ctx* ctx, const double* G_tau, const double* G_bmt, long long c0, long long tc, bool dir,
                  bool need_minus) {
  const long long n = ctx->n, N = ctx->N, nt = ctx->n_tau, ldn = ctx->ldn, nn = n * n, NN = N * N;
  const Split Xt = split3_of(ctx->Xt_h, ctx->Xt_l, ctx->Xt_l2, N, ldn);
  const Split Gs = split3_of(ctx->Gs_h, ctx->Gs_l, ctx->Gs_l2, n, ldn, tc);
  const Split Gms = split3_of(ctx->Gms_h, ctx->Gms_l, ctx->Gms_l2, n, ldn, tc);
  const Split Ys = split3_of(ctx->Ys_h, ctx->Ys_l, ctx->Ys_l2, N, ldn, tc);
  const Split Yms = split3_of(ctx->Yms_h, ctx->Yms_l, ctx->Yms_l2, N, ldn, tc);
  THC_TRY(launch_split_f64(ctx, G_tau + c0 * nn, nn, n, 1, 1.0, Gs, n, "split G"));
  if (G_bmt)
    THC_TRY(launch_split_f64(ctx, G_bmt + c0 * nn, nn, n, 1, -1.0, Gms, n, "split G(-tau)"));
  else
    THC_TRY(launch_split_f64(ctx, G_tau + (nt - 1 - c0) * nn, -nn, n, 1, -1.0, Gms, n, "split G(-tau)"));
  THC_TRY(gemm(ctx, K_PROJECT, Xt, false, Gs, true, N, n, n, tc, EpiSplit<false>{Ys.hi, Ys.lo, ldn, N * ldn, 1.f, Ys.lo2},
               "Y"));
  if (!dir) return THC_OK;
  if (need_minus)
    THC_TRY(gemm(ctx, K_PROJECT, Xt, false, Gms, true, N, n, n, tc,
                 EpiSplit<false>{Yms.hi, Yms.lo, ldn, N * ldn, 1.f, Yms.lo2}, "Ym"));
  // G^X[P][R] = sum_q X^T[P][q] Y[R][q] (X as the three-term A operand)
  THC_TRY(gemm(ctx, K_PROJECT, Xt, false, Ys, true, N, N, n, tc, EpiF32{ctx->GXf, N, NN}, "G^X"));
  if (need_minus)
    THC_TRY(gemm(ctx, K_PROJECT, Xt, false, Yms, true, N, N, n, tc, EpiF32{ctx->GXmf, N, NN}, "G^X(-)"));
  return THC_OK;
}

// Pi from G^X(+-tau) (+ add, FP32) into the split Pi operand, or kept in FP32 (keep).
int split_polarisation(thc_ctx* ctx, long long tc, const float* add, float* keep) {
  const long long N = ctx->N, ldN = ctx->ldN;
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_POLARISATION, 0.0, &rec));
  polarisation_split_kernel<<<blocks_for(tc * N * ldN), 256, 0, ctx->stream>>>(N, tc, ctx->GXf, ctx->GXmf, add, keep,
                                                                               ctx->Pis_h, ctx->Pis_l, ctx->Pis_l2, ldN);
  return prof_end(ctx, &rec, cudaGetLastError(), "polarisation");
}

// D_PR of the chunk from the split Y and G(-tau) of one spin (fused B and C/D, P <= R, mirrored).
int split_sox(thc_ctx* ctx, long long tc) {
  const long long n = ctx->n, N = ctx->N, ldn = ctx->ldn, NN = N * N;
  const Split Gms = split_of(ctx->Gms_h, ctx->Gms_l, n, ldn, tc);
  const Split Ys = split_of(ctx->Ys_h, ctx->Ys_l, N, ldn, tc);
  THC_TRY(check_cuda(ctx, cudaMemsetAsync(ctx->Dd, 0, 8 * tc * NN, ctx->stream), "clear D"));
  const Split U = split_of(ctx->Us_h, ctx->Us_l, N * n, ldn);
  for (long long k = 0; k < tc; ++k) {
    const Split Gmk = Gms.at_batch(k, 1);
    const Split Yk = Ys.at_batch(k, 1);
    double* Dk = ctx->Dd + k * NN;
    for (long long P0 = 0; P0 < N; P0 += ctx->Pb) {
      const long long Pc = std::min<long long>(ctx->Pb, N - P0);
      const Split At = Split{ctx->Ats_h, ctx->Ats_l, n, ldn, Pc, n * ldn};
      // A^T_P[v][q] = sum_s U[P q][s] G(-tau)[v][s]  (G(-tau) carries its sign in Gms)
      THC_TRY(launch_sox_a(ctx, U.at_row(P0 * n, Pc * n), Gmk, At, Pc));
      // D[P][R] += sum_v (sum_w Y[P][w] U[R][v][w]) (sum_q Y[R][q] A^T_P[v][q])  (B and C never stored)
      THC_TRY(launch_bcd(ctx, Yk, U, At, P0, Pc, Dk));
    }
  }
  return launch_mirror_upper(ctx, ctx->Dd, N, tc);  // D_PR = D_RP: fill P > R
}

// Sigma = X M X^T from the split M of the chunk (Ms[b][R][P]).
int split_back(thc_ctx* ctx, long long tc, double* Sigma_chunk) {
  const long long n = ctx->n, N = ctx->N, ldN = ctx->ldN, nn = n * n;
  const Split Xs = split3_of(ctx->Xs_h, ctx->Xs_l, ctx->Xs_l2, n, ldN);
  const Split Ms = split3_of(ctx->Ms_h, ctx->Ms_l, ctx->Ms_l2, N, ldN, tc);
  const Split T2s = split3_of(ctx->T2s_h, ctx->T2s_l, ctx->T2s_l2, n, ldN, tc);
  // T2t[r][R] = sum_P X[r][P] M[R][P]
  THC_TRY(gemm(ctx, K_BACK, Xs, false, Ms, true, n, N, N, tc, EpiSplit<false>{T2s.hi, T2s.lo, ldN, n * ldN, 1.f, T2s.lo2},
               "M X^T"));
  return gemm(ctx, K_BACK, Xs, false, T2s, true, n, n, N, tc, EpiF64{Sigma_chunk, n, nn}, "X T2");
}

// M (merge of D and the direct term with T = V Pi in Ts, or D alone), then Sigma = X M X^T.
int split_merge_back(thc_ctx* ctx, long long tc, bool sox, bool dir, double cd, double* Sigma_chunk) {
  const long long N = ctx->N, ldN = ctx->ldN, NN = N * N;
  const Split Vs = split3_of(ctx->Vs_h, ctx->Vs_l, ctx->Vs_l2, N, ldN);
  const Split Ts = split3_of(ctx->Ts_h, ctx->Ts_l, ctx->Ts_l2, N, ldN, tc);
  const Split Ms = split3_of(ctx->Ms_h, ctx->Ms_l, ctx->Ms_l2, N, ldN, tc);
  if (dir) {
    // W[P][R] = sum_S V[P][S] T[R][S] = (V Pi V)[P][R], symmetric, so the merge epilogue
    // reads the tile as W[R][P]
    THC_TRY(gemm(ctx, K_DIRECT_W, Vs, false, Ts, true, N, N, N, tc,
                 EpiMerge{Ms.hi, Ms.lo, ldN, sox ? ctx->Dd : nullptr, ctx->GXf, (int)N, cd, Ms.lo2}, "W"));
  } else {
    // M[R][P] = c_x D[P][R] = c_x D[R][P] (D mirrored): read along its rows
    THC_TRY(launch_split_f64(ctx, ctx->Dd, NN, N, 1, C_SOX, Ms, N, "split D^T"));
  }
  return split_back(ctx, tc, Sigma_chunk);
}

// Screened direct term (THC_GW) with or without SOX, restricted (nspin 1) or unrestricted
// (nspin 2): the bubble of every tau point from the split projections first (the bosonic
// transform couples them; unrestricted, spin b and then spin a added), the screening in
// FP64 (gw.cu), then per chunk and spin SOX, the merge M = C_SOX D^T - G^X_s o W~ in FP64,
// its split, and the split back-transform.
int split_eval_gw(thc_ctx* ctx, int nspin, const double* const* G_tau, const double* const* G_bmt,
                  double* const* Sigma) {
  const long long n = ctx->n, N = ctx->N, nt = ctx->n_tau, ldN = ctx->ldN, nn = n * n, NN = N * N;
  const bool sox = ctx->terms & THC_SOX;
  if (!ctx->gw_nw) return fail(ctx, THC_EINVAL, "THC_GW needs the bosonic transforms (thc_sigma_set_bosonic)");
  for (long long c0 = 0; c0 < nt; c0 += ctx->tc) {
    const long long tc = std::min<long long>(ctx->tc, nt - c0);
    for (int s = nspin - 1; s >= 0; --s) {
      THC_TRY(split_project(ctx, G_tau[s], G_bmt[s], c0, tc, true, true));
      THC_TRY(gw_store_bubble(ctx, c0, tc, nspin, s));
    }
  }
  THC_TRY(gw_screen(ctx));
  for (long long c0 = 0; c0 < nt; c0 += ctx->tc) {
    const long long tc = std::min<long long>(ctx->tc, nt - c0);
    for (int s = 0; s < nspin; ++s) {
      THC_TRY(split_project(ctx, G_tau[s], G_bmt[s], c0, tc, false, false));  // Y and G(-tau) for SOX
      if (sox) THC_TRY(split_sox(ctx, tc));
      THC_TRY(gw_merge(ctx, c0, tc, sox ? ctx->Dd : nullptr, ctx->gw_m, s));
      const Split Ms = split3_of(ctx->Ms_h, ctx->Ms_l, ctx->Ms_l2, N, ldN, tc);
      THC_TRY(launch_split_f64(ctx, ctx->gw_m, NN, N, 1, 1.0, Ms, N, "split M"));
      THC_TRY(split_back(ctx, tc, Sigma[s] + c0 * nn));
    }
  }
  return THC_OK;
}

}  // namespace

// Restricted (nspin = 1) or unrestricted (nspin = 2) evaluation; the steps and their order
// are those of fp64_eval_spins (THC_GW: split_eval_gw above).  The polarisation of spin b is kept in FP32 (Pif) and added
// to that of spin a before the split of Pi.
int split_eval_spins(thc_ctx* ctx, int nspin, const double* const* G_tau, const double* const* G_bmt,
                     double* const* Sigma) {
  if (ctx->terms & THC_GW) return split_eval_gw(ctx, nspin, G_tau, G_bmt, Sigma);
  const long long n = ctx->n, N = ctx->N, nt = ctx->n_tau, ldN = ctx->ldN, nn = n * n;
  const bool sox = ctx->terms & THC_SOX, dir = ctx->terms & THC_DIRECT;
  const double cd = nspin == 1 ? C_DIRECT : -1.0;
  if (nspin == 2 && dir && !ctx->Pif)
    THC_TRY(ctx_alloc(ctx, (void**)&ctx->Pif, sizeof(float) * (size_t)ctx->tc * N * N, "Pi of spin b"));
  const Split Vs = split3_of(ctx->Vs_h, ctx->Vs_l, ctx->Vs_l2, N, ldN);
  for (long long c0 = 0; c0 < nt; c0 += ctx->tc) {
    const long long tc = std::min<long long>(ctx->tc, nt - c0);
    const Split Pis = split3_of(ctx->Pis_h, ctx->Pis_l, ctx->Pis_l2, N, ldN, tc);
    const Split Ts = split3_of(ctx->Ts_h, ctx->Ts_l, ctx->Ts_l2, N, ldN, tc);
    if (nspin == 2 && dir) {
      THC_TRY(split_project(ctx, G_tau[1], G_bmt[1], c0, tc, true, true));
      THC_TRY(split_polarisation(ctx, tc, nullptr, ctx->Pif));
    }
    THC_TRY(split_project(ctx, G_tau[0], G_bmt[0], c0, tc, dir, true));
    if (dir) {
      THC_TRY(split_polarisation(ctx, tc, nspin == 2 ? ctx->Pif : nullptr, nullptr));
      THC_TRY(gemm(ctx, K_DIRECT_VPI, Vs, false, Pis, true, N, N, N, tc,
                   EpiSplit<false>{Ts.hi, Ts.lo, ldN, N * ldN, 1.f, Ts.lo2}, "V Pi"));
    }
    for (int s = 0; s < nspin; ++s) {
      if (s == 1) THC_TRY(split_project(ctx, G_tau[1], G_bmt[1], c0, tc, dir, false));
      if (sox) THC_TRY(split_sox(ctx, tc));
      THC_TRY(split_merge_back(ctx, tc, sox, dir, cd, Sigma[s] + c0 * nn));
    }
  }
  return THC_OK;
}

int split_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, double* Sigma) {
  return split_eval_spins(ctx, 1, &G_tau, &G_bmt, &Sigma);
}

// ------------------------------------------------------- autotuner cache
// Text file, one shape per line: kclass M N K batch choice (the tile width 128 / 256 of a
// single-chunk contraction, or the cluster shape 10 CP + CR of a fused B C/D block, whose
// "batch" field is the block's first P).
int autotune_save(const char* path) {
  std::lock_guard<std::mutex> lock(g_tile_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(nullptr, THC_EINVAL, std::string("cannot write ") + path);
  for (const auto& kv : g_tile_table)
    std::fprintf(f, "%d %lld %lld %lld %lld %d\n", kv.first.kclass, kv.first.M, kv.first.N, kv.first.K,
                 kv.first.batch, kv.second);
  std::fclose(f);
  return THC_OK;
}

int autotune_load(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(nullptr, THC_EINVAL, std::string("cannot read ") + path);
  std::lock_guard<std::mutex> lock(g_tile_mu);
  ShapeKey k;
  int bn;
  while (std::fscanf(f, "%d %lld %lld %lld %lld %d", &k.kclass, &k.M, &k.N, &k.K, &k.batch, &bn) == 6)
    if (k.kclass == K_SOX_BCD ? (bn == 11 || bn == 12 || bn == 22) : (bn == 128 || bn == 256)) g_tile_table[k] = bn;
  std::fclose(f);
  return THC_OK;
}

int autotune_entries() {
  std::lock_guard<std::mutex> lock(g_tile_mu);
  return (int)g_tile_table.size();
}

// --------------------------------------------------- standalone utility
int gemm_bf16x3(cudaStream_t stream, int batch, int M, int N, int K, const double* A, long long sA, const double* B,
                long long sB, double* C, long long sC) {
  thc_ctx tmp;
  tmp.stream = stream;
  THC_TRY(get_encoder(nullptr));
  const long long ldK = pad8(K);
  const long long ba = sA ? batch : 1, bb = sB ? batch : 1;
  const size_t h = sizeof(bf16);
  void *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr, *err = nullptr;
  auto cleanup = [&]() {
    if (ah) cudaFreeAsync(ah, stream);
    if (al) cudaFreeAsync(al, stream);
    if (bh) cudaFreeAsync(bh, stream);
    if (bl) cudaFreeAsync(bl, stream);
    if (err) cudaFreeAsync(err, stream);
  };
  auto alloc = [&](void** p, size_t bytes) { return cudaMallocAsync(p, std::max<size_t>(bytes, 16), stream); };
  if (alloc(&ah, h * ba * M * ldK) || alloc(&al, h * ba * M * ldK) || alloc(&bh, h * bb * N * ldK) ||
      alloc(&bl, h * bb * N * ldK) || alloc(&err, 2 * sizeof(int))) {
    cudaGetLastError();
    cleanup();
    return fail(nullptr, THC_ENOMEM, "thc_gemm_bf16x3: allocation failed");
  }
  tmp.d_err = (int*)err;
  int rc = check_cuda(nullptr, cudaMemsetAsync(err, 0, 2 * sizeof(int), stream), "thc_gemm_bf16x3: clear flag");
  const Split As = Split{(bf16*)ah, (bf16*)al, M, ldK, ba, (long long)M * ldK};
  const Split Bs = Split{(bf16*)bh, (bf16*)bl, N, ldK, bb, (long long)N * ldK};
  if (rc == THC_OK) rc = launch_split_f64(&tmp, A, sA, K, 1, 1.0, As, K, "split A");
  if (rc == THC_OK) rc = launch_split_f64(&tmp, B, sB, K, 1, 1.0, Bs, K, "split B");
  if (rc == THC_OK)
    rc = gemm(&tmp, K_BACK, As, ba > 1, Bs, bb > 1, M, N, K, batch, EpiF64{C, N, sC}, "thc_gemm_bf16x3");
  if (rc == THC_OK) rc = status_check(&tmp);
  cleanup();
  cudaStreamSynchronize(stream);
  if (rc != THC_OK) fail(nullptr, rc, tmp.err);
  return rc;
}

}  // namespace thc
