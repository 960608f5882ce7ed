// FP64 register-tiled contraction machinery (DFMA).
//
// On GB300 FP64 runs at about 2 fused multiply-adds per clock per SM
// (1.19 TFLOP/s measured for the whole GPU), three orders of magnitude below
// the BF16 tensor rate, and no FP64 tcgen05 kind exists.  A FP64 contraction
// is therefore bound by the DFMA pipe alone: the tile below keeps 16
// independent accumulators per thread, stages operands through shared memory
// with plain coalesced loads, and skips the multiply-adds of warps whose
// 16 x 32 sub-tile lies wholly outside the matrix so that ragged edges cost
// little DFMA time.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace thc {
namespace f64 {

constexpr int BM = 64;   // rows of a CTA tile (m)
constexpr int BN = 64;   // columns of a CTA tile (n)
constexpr int BK = 16;   // depth of one shared-memory stage (k)
constexpr int NT = 256;  // threads: 8 warps = 4 (m) x 2 (n); warp tile 16 x 32; lane tile 4 x 4
constexpr int LDS = BM + 2;  // padded row of a shared tile (16-byte aligned rows)

// Strided batched matrix view: element (b, r, c) at p[b*sb + r*sr + c*sc].
struct View {
  const double* p;
  long long sb, sr, sc;
  __device__ __forceinline__ double at(long long b, long long r, long long c) const {
    return p[b * sb + r * sr + c * sc];
  }
};

// Khatri-Rao operand of the U build: B(k = Q, n = q*n + s) = X_qQ X_sQ, generated on the fly.
struct KhatriRao {
  const double* X;  // n x N row-major
  int n, N;
  __device__ __forceinline__ double at(long long, long long k, long long c) const {
    const long long q = c / n, s = c - q * n;
    return X[q * N + k] * X[s * N + k];
  }
};

struct Tiles {
  double A[BK][LDS];  // A[k][m]
  double B[BK][LDS];  // B[k][n]
};

// Load an A tile (rows m0.., depth k0..) into T.A[k][m]; zero outside (M, K).
// KFAST: consecutive threads walk k (operand contiguous along k); else along m.
template <bool KFAST, class L>
__device__ __forceinline__ void load_a(Tiles& T, const L& a, long long b, long long m0, long long k0,
                                       long long M, long long K) {
  const int t = threadIdx.x;
  if (KFAST) {
    const int k = t & 15, mm = t >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = mm + 16 * i;
      T.A[k][m] = (m0 + m < M && k0 + k < K) ? a.at(b, m0 + m, k0 + k) : 0.0;
    }
  } else {
    const int m = t & 63, kk = t >> 6;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = kk + 4 * i;
      T.A[k][m] = (m0 + m < M && k0 + k < K) ? a.at(b, m0 + m, k0 + k) : 0.0;
    }
  }
}

// Load a B tile (depth k0.., columns n0..) into T.B[k][n]; zero outside (K, Nn).
template <bool KFAST, class L>
__device__ __forceinline__ void load_b(Tiles& T, const L& bop, long long b, long long k0, long long n0,
                                       long long K, long long Nn) {
  const int t = threadIdx.x;
  if (KFAST) {
    const int k = t & 15, nn = t >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = nn + 16 * i;
      T.B[k][c] = (k0 + k < K && n0 + c < Nn) ? bop.at(b, k0 + k, n0 + c) : 0.0;
    }
  } else {
    const int c = t & 63, kk = t >> 6;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = kk + 4 * i;
      T.B[k][c] = (k0 + k < K && n0 + c < Nn) ? bop.at(b, k0 + k, n0 + c) : 0.0;
    }
  }
}

// Thread coordinates inside the CTA tile.
struct Lane {
  int rm, rn;  // first row / column of the thread's 4 x 4 sub-tile
  int wm, wn;  // warp coordinates
  int lm, ln;  // lane coordinates within the warp
  __device__ __forceinline__ Lane() {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    wm = warp & 3;
    wn = warp >> 2;
    lm = lane >> 3;
    ln = lane & 7;
    rm = wm * 16 + lm * 4;
    rn = wn * 32 + ln * 4;
  }
};

// acc += A[m0:m0+BM, :K] * B[:K, n0:n0+BN] for batch b.
template <bool AK, bool BK_, class LA, class LB>
__device__ __forceinline__ void mainloop(Tiles& T, const LA& la, const LB& lb, long long b, long long m0,
                                         long long n0, long long M, long long Nn, long long K,
                                         const Lane& L, double (&acc)[4][4]) {
  const bool active = (m0 + L.wm * 16 < M) && (n0 + L.wn * 32 < Nn);
  for (long long k0 = 0; k0 < K; k0 += BK) {
    load_a<AK>(T, la, b, m0, k0, M, K);
    load_b<BK_>(T, lb, b, k0, n0, K, Nn);
    __syncthreads();
    if (active) {
      const long long rem = K - k0;
      if (rem >= BK) {
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          const double2 a01 = *reinterpret_cast<const double2*>(&T.A[kk][L.rm]);
          const double2 a23 = *reinterpret_cast<const double2*>(&T.A[kk][L.rm + 2]);
          const double2 b01 = *reinterpret_cast<const double2*>(&T.B[kk][L.rn]);
          const double2 b23 = *reinterpret_cast<const double2*>(&T.B[kk][L.rn + 2]);
          const double av[4] = {a01.x, a01.y, a23.x, a23.y};
          const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
      } else {
        for (int kk = 0; kk < (int)rem; ++kk) {
          double av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = T.A[kk][L.rm + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = T.B[kk][L.rn + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
      }
    }
    __syncthreads();
  }
}

// Plain store epilogue: C(b, m, n) = alpha * acc.
struct StoreEpi {
  double* p;
  long long sb, sr, sc;
  double alpha;
  __device__ __forceinline__ void operator()(long long b, long long m, long long c, double v) const {
    p[b * sb + m * sr + c * sc] = alpha * v;
  }
};

// Store epilogue of a contraction whose batch b needs only the columns c >= c0 + b
// (the rest lies below the diagonal of a symmetric result): tiles wholly left of
// that bound are not computed.
struct TriStoreEpi {
  double* p;
  long long sb, sr, sc;
  double alpha;
  long long c0;
  __device__ __forceinline__ void operator()(long long b, long long m, long long c, double v) const {
    p[b * sb + m * sr + c * sc] = alpha * v;
  }
  __device__ __forceinline__ bool skip_tile(long long b, long long, long long c_end) const { return c_end <= c0 + b; }
};

template <class E, class = void>
struct HasSkipTile : std::false_type {};
template <class E>
struct HasSkipTile<E, std::void_t<decltype(&E::skip_tile)>> : std::true_type {};

// Generic batched contraction: C(b) = epi(A(b) B(b)); grid (ceil(M/BM), ceil(Nn/BN), batch).
// An epilogue with skip_tile(b, m0, c_end) drops whole CTA tiles (rows m0 .., columns
// below c_end) it does not need.
template <bool AK, bool BK_, class LA, class LB, class Epi>
__global__ void __launch_bounds__(NT) gemm_kernel(long long M, long long Nn, long long K, LA la, LB lb,
                                                  Epi epi) {
  __shared__ __align__(16) Tiles T;
  const long long b = blockIdx.z;
  const long long m0 = (long long)blockIdx.x * BM, n0 = (long long)blockIdx.y * BN;
  if constexpr (HasSkipTile<Epi>::value) {
    if (epi.skip_tile(b, m0, n0 + BN)) return;
  }
  const Lane L;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  mainloop<AK, BK_>(T, la, lb, b, m0, n0, M, Nn, K, L, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long m = m0 + L.rm + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long c = n0 + L.rn + j;
      if (c < Nn) epi(b, m, c, acc[i][j]);
    }
  }
}

}  // namespace f64
}  // namespace thc
