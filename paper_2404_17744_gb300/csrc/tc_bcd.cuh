// Fused B and C/D contractions of the SOX term (Sec. II.C) in split precision
// on the 5th-generation tensor cores (sm_103a), for one tau point and one
// block of P:
//
//   C_v[P][R] = sum_w Y[P0 + P][w] U[R][v][w]           (C_RvP of the scheme)
//   B_v[P][R] = sum_q A^T[P][v][q] Y[R][q]              (B_PRv)
//   D[P0 + P][R] += sum_v C_v[P][R] B_v[P][R]           (D_PR)
//
// For a fixed v both products are 128 x 128 tiles with the same layout (TMEM
// lane = P, column = R), so one CTA computes C_v and B_v of its (P, R) tile
// into TMEM and the epilogue multiplies them in registers and accumulates the
// tile of D over v.  Neither B nor C is ever stored: compared with writing B
// in FP32 and reading it back in the C/D step this removes 8 N^2 n bytes of
// HBM traffic per tau point and block, and the tiles carry no padding along
// v (v is the loop index, not a tile dimension).
//
// Work units are (P tile, R tile, v chunk); the v range of a (P, R) tile is cut
// into chunks so that the units fill the SMs in whole waves, and every unit adds
// its FP32 partial tile of D into the FP64 D with one atomic per element.  Units
// are numbered with the v chunk slowest, so the CTAs of a wave walk the same few
// values of v together and the U_v and A^T_v slices they read are served from
// L2.  A persistent CTA takes units blockIdx.x, blockIdx.x + gridDim.x, ...
//
// Warp roles (as in split_gemm_kernel):
//   warp 0    one lane issues the TMA loads of every 64-deep K stage: for the C
//             product Y rows of the P tile and the U_v rows of the R tile, for
//             the B product the A^T_v rows of the P tile and Y rows of the R tile
//             (hi and lo halves of both operands, 128-byte swizzle);
//   warp 1    allocates 512 TMEM columns (two buffers of [C_v | B_v]); one lane
//             issues the 3 x 4 tcgen05.mma per stage (hi hi, hi lo, lo hi) of
//             both products of one v into one buffer, so the MMAs of v + 1 run
//             while the epilogue reads v;
//   warps 2-9 read C_v and B_v of their 32 lanes x 64 columns with tcgen05.ld,
//             accumulate the products in FP32 registers, and at the end of a
//             unit add the tile to D through a per-warp swizzled 32 x 32 staging
//             tile (lanes along R: coalesced FP64 atomics).
// Every wait is bounded in time; a wait that runs out sets *err and the CTA
// unwinds.
#pragma once

#include "tc_gemm.cuh"

namespace thc {
namespace tc {

struct BcdCfg {
  static constexpr int OP = BM * BKE * 2;          // one 128 x 64 BF16 operand block, 16 KB
  static constexpr int STAGE = 4 * OP;             // A hi, A lo, B hi, B lo
  static constexpr int STAGES = 3;
  static constexpr int STAGING = 8 * 32 * 32 * 4;  // one 32 x 32 FP32 flush tile per epilogue warp
  static constexpr int SMEM = STAGES * STAGE + STAGING + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int TMEM_COLS = 512;            // buffer b: C_v at 256 b, B_v at 256 b + 128
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

struct BcdArgs {
  int Pc;     // rows of the P block (A^T has Pc rows, D rows P0 .. P0 + Pc - 1)
  int P0;     // first P of the block: row offset into Y and D
  int N;      // THC rank: range of R, rows of Y, row length of D
  int n;      // AO count: range of v, depth (w, q) of both products
  int nvc;    // v chunks per (P, R) tile
  double* D;  // N x N FP64, D[P][R] at P * N + R
};

// Maps: Y (k, row, 1), box 64 x 128 x 1; U (w, v, R) and A^T (q, v, P), box 64 x 1 x 128.
__global__ void __launch_bounds__(NTHREADS, 1)
    sox_bcd_kernel(const __grid_constant__ CUtensorMap mYhi, const __grid_constant__ CUtensorMap mYlo,
                   const __grid_constant__ CUtensorMap mUhi, const __grid_constant__ CUtensorMap mUlo,
                   const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo, BcdArgs a,
                   int* err) {
  using C = BcdCfg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* staging = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE + C::STAGING);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;  // [2] C_v and B_v of a v ready
  uint64_t* acc_free = acc_full + 2;       // [2] buffer read by the epilogue
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_free + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (a.n + BKE - 1) / BKE;
  const int tm = (a.Pc + BM - 1) / BM, tn = (a.N + BM - 1) / BM;
  const long long tiles = (long long)tm * tn, units = tiles * a.nvc;
  // unit u: v chunk u / tiles (slowest), then P tile fastest
  auto decode = [&](long long u, int& pt, int& rt, int& v0, int& v1) {
    const long long vc = u / tiles, t = u - vc * tiles;
    pt = (int)(t % tm);
    rt = (int)(t / tm);
    v0 = (int)(vc * a.n / a.nvc);
    v1 = (int)((vc + 1) * a.n / a.nvc);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_free[i], NEPI);
    }
    fence_mbar_init();
    prefetch_map(&mYhi);
    prefetch_map(&mYlo);
    prefetch_map(&mUhi);
    prefetch_map(&mUlo);
    prefetch_map(&mAhi);
    prefetch_map(&mAlo);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;  // running K-stage counter
      bool ok = true;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        int pt, rt, v0, v1;
        decode(u, pt, rt, v0, v1);
        for (int v = v0; v < v1 && ok; ++v) {
          for (int prod = 0; prod < 2 && ok; ++prod) {
            for (int kb = 0; kb < nkb; ++kb, ++g) {
              const int s = (int)(g % C::STAGES);
              const uint32_t r = (uint32_t)(g / C::STAGES);
              if (!mbar_wait(&empty[s], (r & 1) ^ 1)) {
                atomicExch(err, 11);
                ok = false;
                break;
              }
              uint8_t* st = smem + s * C::STAGE;
              const int k0 = kb * BKE;
              mbar_arrive_expect_tx(&full[s], C::STAGE);
              if (prod == 0) {  // C_v: A = Y (P tile), B = U_v (R tile)
                tma_load_3d(st, &mYhi, &full[s], k0, a.P0 + pt * BM, 0);
                tma_load_3d(st + C::OP, &mYlo, &full[s], k0, a.P0 + pt * BM, 0);
                tma_load_3d(st + 2 * C::OP, &mUhi, &full[s], k0, v, rt * BM);
                tma_load_3d(st + 3 * C::OP, &mUlo, &full[s], k0, v, rt * BM);
              } else {          // B_v: A = A^T_v (P tile), B = Y (R tile)
                tma_load_3d(st, &mAhi, &full[s], k0, v, pt * BM);
                tma_load_3d(st + C::OP, &mAlo, &full[s], k0, v, pt * BM);
                tma_load_3d(st + 2 * C::OP, &mYhi, &full[s], k0, rt * BM, 0);
                tma_load_3d(st + 3 * C::OP, &mYlo, &full[s], k0, rt * BM, 0);
              }
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0, j = 0;  // K stages and v steps handled by this CTA
      bool ok = true;
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        int pt, rt, v0, v1;
        decode(u, pt, rt, v0, v1);
        // a ragged last R tile multiplies only its round-up-to-16 width
        const uint32_t idesc = idesc_bf16(BM, min(BM, (a.N - rt * BM + 15) & ~15));
        for (int v = v0; v < v1 && ok; ++v, ++j) {
          const int buf = (int)(j & 1);
          if (!mbar_wait(&acc_free[buf], ((uint32_t)(j >> 1) & 1) ^ 1)) {
            atomicExch(err, 12);
            ok = false;
            break;
          }
          tc_fence_after();
          for (int prod = 0; prod < 2 && ok; ++prod) {
            const uint32_t d = tmem + static_cast<uint32_t>(buf * 256 + prod * 128);
            for (int kb = 0; kb < nkb; ++kb, ++g) {
              const int s = (int)(g % C::STAGES);
              if (!mbar_wait(&full[s], (uint32_t)(g / C::STAGES) & 1)) {
                atomicExch(err, 12);
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t base = smem_u32(smem + s * C::STAGE);
              const uint64_t ah = sw128_desc(base), al = sw128_desc(base + C::OP);
              const uint64_t bh = sw128_desc(base + 2 * C::OP), bl = sw128_desc(base + 3 * C::OP);
              const int ksteps = min(BKE / 16, (a.n - kb * BKE + 15) >> 4);
#pragma unroll
              for (int k = 0; k < BKE / 16; ++k) {
                if (k < ksteps) {
                  const uint64_t off = static_cast<uint64_t>((k * 32) >> 4);  // 16 BF16 = 32 bytes along K
                  mma_bf16(d, ah + off, bh + off, idesc, (kb | k) != 0);
                  mma_bf16(d, ah + off, bl + off, idesc, 1u);
                  mma_bf16(d, al + off, bh + off, idesc, 1u);
                }
              }
              mma_commit(&empty[s]);
            }
          }
          if (ok) mma_commit(&acc_full[buf]);  // C_v and B_v of this v complete
        }
      }
    }
  } else {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + half * 64;
    const TileRef tile{staging + (warp - 2) * 32 * 32};
    long long j = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
      int pt, rt, v0, v1;
      decode(u, pt, rt, v0, v1);
      float acc[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) acc[i] = 0.f;
      for (int v = v0; v < v1; ++v, ++j) {
        const int buf = (int)(j & 1);
        if (!mbar_wait(&acc_full[buf], (uint32_t)(j >> 1) & 1)) {
          if (lane == 0) atomicExch(err, 13);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t src = lane_base + buf * 256;
#pragma unroll
        for (int c = 0; c < 64; c += 32) {
          uint32_t cv[32], bv[32];
          tmem_ld16(src + c, cv);
          tmem_ld16(src + c + 16, cv + 16);
          tmem_ld16(src + 128 + c, bv);
          tmem_ld16(src + 128 + c + 16, bv + 16);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[c + i] = fmaf(__uint_as_float(cv[i]), __uint_as_float(bv[i]), acc[c + i]);
        }
        tc_fence_before();
        mbar_arrive(&acc_free[buf]);
      }
      if (!ok) break;
      // D[P0 + P][R] += acc: lane r of the warp holds row P = pt 128 + quarter 32 + r
      const int prow = pt * BM + quarter * 32;
#pragma unroll
      for (int c = 0; c < 64; c += 32) {
#pragma unroll
        for (int i = 0; i < 32; ++i) tile(lane, i) = acc[c + i];
        __syncwarp();
        const int R = rt * BM + half * 64 + c + lane;
        if (R < a.N) {
          for (int r = 0; r < 32 && prow + r < a.Pc; ++r)
            atomicAdd(&a.D[(long long)(a.P0 + prow + r) * a.N + R], (double)tile(r, lane));
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

}  // namespace tc
}  // namespace thc
