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
// its FP32 partial tile of D into the FP64 D with one atomic per element.  D_PR is
// symmetric for symmetric G(+-tau) (rename w <-> q, v <-> s and use U_Pqs = U_Psq),
// so only tiles that reach R >= P are computed, only P <= R is added, and the
// caller mirrors the rest.  Units
// are numbered with the v chunk slowest, so the CTAs of a wave walk the same few
// values of v together and the U_v and A^T_v slices they read are served from
// L2.  A persistent cluster takes units c, c + clusters, ...
//
// CTAs run in clusters of CP x CR (1 x 2 in use): the CTAs of a cluster share
// their P tile (or R tile) and so the operands of that side.  Each loads one
// slice of a shared operand block and multicasts it (TMA .multicast::cluster)
// to the CTAs that need it, which cuts the operand traffic from L2 by a quarter
// for a pair along R.
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
  int nvc;    // v chunks per cluster tile
  int tail;   // 16 or 32: the last K block of both products (n mod 64 <= tail, n > 64) is
              // loaded with boxes that wide into one shared stage; 0: every K block alone
  double* D;  // N x N FP64, D[P][R] at P * N + R
};

// Tensor maps of one operand half (hi or lo): Y rows for the P side (box 64 x 128/CR)
// and the R side (box 64 x 128/CP), U (w, v, R) with box 64 x 1 x 128/CP, and
// A^T (q, v, P) with box 64 x 1 x 128/CR; the same four with boxes of the tail width.
struct BcdMaps {
  CUtensorMap yp, yr, u, at;
  CUtensorMap ypt, yrt, ut, att;
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n barrier.cluster.wait.acquire;" ::: "memory");
}
// TMA load of a box into the same shared-memory offset of every CTA in mask, each
// of whose mbarrier at offset bar receives the completed bytes.
__device__ __forceinline__ void tma_load_3d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                               int c2, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster [%0], "
      "[%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}
// tcgen05.commit arriving on the mbarrier at offset bar of every CTA in mask.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// CP x CR cluster (rank = pi CR + rj) over a (CP 128) x (CR 128) block of D:
// CTA (pi, rj) owns P tile CP t_P + pi and R tile CR t_R + rj.  The P-side operands
// (Y rows of the P tile, A^T_v) are common to the CR CTAs of a row pi: each loads
// one 128/CR-row slice and multicasts it to them; the R-side operands (U_v, Y rows
// of the R tile) likewise across the CP CTAs of a column rj.  Every CTA's MMA
// releases a stage on all CTAs of the cluster, so a producer refills a stage only
// when every CTA it writes into has consumed it.  CP = CR = 1 is the plain kernel.
template <int CP, int CR>
__global__ void __launch_bounds__(NTHREADS, 1)
    sox_bcd_kernel(const __grid_constant__ BcdMaps hi, const __grid_constant__ BcdMaps lo, BcdArgs a, int* err) {
  using C = BcdCfg;
  constexpr int CS = CP * CR;
  constexpr int PROWS = BM / CR, RROWS = BM / CP;  // rows of the slices this CTA loads
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* staging = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE + C::STAGING);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;  // [2] C_v and B_v of a v ready
  uint64_t* acc_free = acc_full + 2;       // [2] buffer read by the epilogue
  uint64_t* drain = acc_free + 2;          // every MMA of this CTA complete (unwind)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = CS > 1 ? cluster_ctarank() : 0u;
  const int pi = (int)rank / CR, rj = (int)rank % CR;
  const int nkb = (a.n + BKE - 1) / BKE;
  // K blocks each product loads alone; with a tail, its last block shares one stage with the
  // other product's (8 narrow blocks: C's Y_P and U_v, B's A^T_v and Y_R, hi and lo)
  const int nkf = a.tail ? nkb - 1 : nkb;
  const int NB = BM * 2 * a.tail;  // bytes of one narrow block
  const int tk0 = (nkb - 1) * BKE;  // first K of the tail
  const int tm = (a.Pc + BM - 1) / BM, tn = (a.N + BM - 1) / BM;
  const int tm2 = (tm + CP - 1) / CP, tn2 = (tn + CR - 1) / CR;
  // D is symmetric: only cluster tiles that reach R >= P are computed.  Cluster row i
  // (P from P0 + i CP 128) starts at cluster column first_col(i); ctiles counts them.
  auto first_col = [&](int i) { return (int)((a.P0 + (long long)i * CP * BM) / ((long long)CR * BM)); };
  long long ctiles = 0;
  for (int i = 0; i < tm2; ++i) ctiles += max(0, tn2 - first_col(i));
  const long long units = ctiles * a.nvc;
  const long long cl = blockIdx.x / CS, ncl = gridDim.x / CS;
  // unit u of a cluster: v chunk u / ctiles (slowest), then the upper cluster tiles row by row
  auto decode = [&](long long u, int& pt, int& rt, int& v0, int& v1) {
    const long long vc = u / ctiles;
    long long t = u - vc * ctiles;
    int i = 0;
    for (; i < tm2; ++i) {
      const int c = max(0, tn2 - first_col(i));
      if (t < c) break;
      t -= c;
    }
    pt = i * CP + pi;
    rt = (first_col(i) + (int)t) * CR + rj;
    v0 = (int)(vc * a.n / a.nvc);
    v1 = (int)((vc + 1) * a.n / a.nvc);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CS);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_free[i], NEPI);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
    prefetch_map(&hi.yp);
    prefetch_map(&lo.yp);
    prefetch_map(&hi.yr);
    prefetch_map(&lo.yr);
    prefetch_map(&hi.u);
    prefetch_map(&lo.u);
    prefetch_map(&hi.at);
    prefetch_map(&lo.at);
    if (a.tail) {
      prefetch_map(&hi.ypt);
      prefetch_map(&lo.ypt);
      prefetch_map(&hi.yrt);
      prefetch_map(&lo.yrt);
      prefetch_map(&hi.ut);
      prefetch_map(&lo.ut);
      prefetch_map(&hi.att);
      prefetch_map(&lo.att);
    }
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CS > 1) cluster_sync_all();  // every CTA's barriers exist before any multicast
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint16_t pmask = 0, rmask = 0;  // CTAs sharing this CTA's P tile / R tile
      for (int r = 0; r < CR; ++r) pmask |= (uint16_t)(1u << (pi * CR + r));
      for (int p = 0; p < CP; ++p) rmask |= (uint16_t)(1u << (p * CR + rj));
      // one slice of an operand block (rows of rowb bytes): multicast when shared, a plain
      // load otherwise
      auto load = [&](uint8_t* blk, int slice, int rows, const CUtensorMap* m, uint64_t* bar, int c0, int c1, int c2,
                      uint16_t mask, bool shared, int rowb = 128) {
        uint8_t* dst = blk + slice * rows * rowb;
        if (shared)
          tma_load_3d_mc(dst, m, bar, c0, c1, c2, mask);
        else
          tma_load_3d(dst, m, bar, c0, c1, c2);
      };
      long long g = 0;  // running K-stage counter
      bool ok = true;
      for (long long u = cl; u < units && ok; u += ncl) {
        int pt, rt, v0, v1;
        decode(u, pt, rt, v0, v1);
        const int prow = pt * BM + rj * PROWS, rrow = rt * BM + pi * RROWS;  // first rows of this CTA's slices
        for (int v = v0; v < v1 && ok; ++v) {
          for (int prod = 0; prod < 2 && ok; ++prod) {
            for (int kb = 0; kb < nkf; ++kb, ++g) {
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
                load(st, rj, PROWS, &hi.yp, &full[s], k0, a.P0 + prow, 0, pmask, CR > 1);
                load(st + C::OP, rj, PROWS, &lo.yp, &full[s], k0, a.P0 + prow, 0, pmask, CR > 1);
                load(st + 2 * C::OP, pi, RROWS, &hi.u, &full[s], k0, v, rrow, rmask, CP > 1);
                load(st + 3 * C::OP, pi, RROWS, &lo.u, &full[s], k0, v, rrow, rmask, CP > 1);
              } else {          // B_v: A = A^T_v (P tile), B = Y (R tile)
                load(st, rj, PROWS, &hi.at, &full[s], k0, v, prow, pmask, CR > 1);
                load(st + C::OP, rj, PROWS, &lo.at, &full[s], k0, v, prow, pmask, CR > 1);
                load(st + 2 * C::OP, pi, RROWS, &hi.yr, &full[s], k0, rrow, 0, rmask, CP > 1);
                load(st + 3 * C::OP, pi, RROWS, &lo.yr, &full[s], k0, rrow, 0, rmask, CP > 1);
              }
            }
          }
          if (a.tail && ok) {  // the tails of both products in one stage
            const int s = (int)(g % C::STAGES);
            const uint32_t r = (uint32_t)(g / C::STAGES);
            if (!mbar_wait(&empty[s], (r & 1) ^ 1)) {
              atomicExch(err, 11);
              ok = false;
              break;
            }
            uint8_t* st = smem + s * C::STAGE;
            const int rb = 2 * a.tail;
            mbar_arrive_expect_tx(&full[s], (uint32_t)(8 * NB));
            load(st, rj, PROWS, &hi.ypt, &full[s], tk0, a.P0 + prow, 0, pmask, CR > 1, rb);
            load(st + NB, rj, PROWS, &lo.ypt, &full[s], tk0, a.P0 + prow, 0, pmask, CR > 1, rb);
            load(st + 2 * NB, pi, RROWS, &hi.ut, &full[s], tk0, v, rrow, rmask, CP > 1, rb);
            load(st + 3 * NB, pi, RROWS, &lo.ut, &full[s], tk0, v, rrow, rmask, CP > 1, rb);
            load(st + 4 * NB, rj, PROWS, &hi.att, &full[s], tk0, v, prow, pmask, CR > 1, rb);
            load(st + 5 * NB, rj, PROWS, &lo.att, &full[s], tk0, v, prow, pmask, CR > 1, rb);
            load(st + 6 * NB, pi, RROWS, &hi.yrt, &full[s], tk0, rrow, 0, rmask, CP > 1, rb);
            load(st + 7 * NB, pi, RROWS, &lo.yrt, &full[s], tk0, rrow, 0, rmask, CP > 1, rb);
            ++g;
          }
        }
      }
      // every copy this CTA armed has landed before it may leave (immediate unless a wait ran out)
      if (!drain_stages(full, C::STAGES, g)) atomicExch(err, 15);
      if constexpr (CS > 1) {
        // every CTA's release of the last stages has arrived here before the CTA can exit
        for (int i = 0; i < C::STAGES && ok; ++i, ++g) {
          if (!mbar_wait(&empty[g % C::STAGES], ((uint32_t)(g / C::STAGES) & 1) ^ 1)) {
            atomicExch(err, 14);
            ok = false;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint16_t all = (uint16_t)((1u << CS) - 1);
      long long g = 0, j = 0;  // K stages and v steps handled by this CTA
      bool ok = true;
      for (long long u = cl; u < units && ok; u += ncl) {
        int pt, rt, v0, v1;
        decode(u, pt, rt, v0, v1);
        // a ragged last R tile multiplies only its round-up-to-16 width (at least 16)
        const uint32_t idesc = idesc_bf16(BM, max(16, min(BM, (a.N - rt * BM + 15) & ~15)));
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
            for (int kb = 0; kb < nkf; ++kb, ++g) {
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
              if constexpr (CS > 1)
                mma_commit_mc(&empty[s], all);  // the stage is free here and in every CTA loading into it
              else
                mma_commit(&empty[s]);
            }
          }
          if (a.tail && ok) {  // the tails of C_v and B_v from the shared stage (accumulating)
            const int s = (int)(g % C::STAGES);
            if (!mbar_wait(&full[s], (uint32_t)(g / C::STAGES) & 1)) {
              atomicExch(err, 12);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * C::STAGE);
            const int ksteps = (a.n - tk0 + 15) >> 4;  // 1 or 2 for a tail of 16 or 32
            for (int prod = 0; prod < 2; ++prod) {
              const uint32_t d = tmem + static_cast<uint32_t>(buf * 256 + prod * 128);
              const uint32_t b0 = base + (uint32_t)(4 * prod * NB);
              const uint64_t ah = narrow_desc(b0, a.tail), al = narrow_desc(b0 + NB, a.tail);
              const uint64_t bh = narrow_desc(b0 + 2 * NB, a.tail), bl = narrow_desc(b0 + 3 * NB, a.tail);
              for (int k = 0; k < ksteps; ++k) {
                const uint64_t off = static_cast<uint64_t>((k * 32) >> 4);
                mma_bf16(d, ah + off, bh + off, idesc, 1u);
                mma_bf16(d, ah + off, bl + off, idesc, 1u);
                mma_bf16(d, al + off, bh + off, idesc, 1u);
              }
            }
            if constexpr (CS > 1)
              mma_commit_mc(&empty[s], all);
            else
              mma_commit(&empty[s]);
            ++g;
          }
          if (ok) mma_commit(&acc_full[buf]);  // C_v and B_v of this v complete
        }
      }
      // every MMA issued (and the barrier arrivals it signals in the cluster) has completed
      // before TMEM is freed (immediate unless a wait ran out)
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicExch(err, 16);
    }
  } else {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + half * 64;
    const TileRef tile{staging + (warp - 2) * 32 * 32};
    long long j = 0;
    bool ok = true;
    for (long long u = cl; u < units && ok; u += ncl) {
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
        if (R < a.N) {  // the upper triangle only: P0 + P <= R
          for (int r = 0; r < 32 && prow + r < a.Pc && a.P0 + prow + r <= R; ++r)
            atomicAdd(&a.D[(long long)(a.P0 + prow + r) * a.N + R], (double)tile(r, lane));
        }
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CS > 1) cluster_sync_all();  // no CTA leaves while another may still signal it
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

}  // namespace tc
}  // namespace thc
