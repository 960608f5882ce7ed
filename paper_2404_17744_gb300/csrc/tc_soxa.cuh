// SOX contraction A of the scheme (Sec. II.C) in split precision on the 5th-generation
// tensor cores (sm_103a), for one tau point and one block of P:
//
//   A^T[P][v][q] = sum_s U[P][q][s] G(-tau)[v][s]         (A_Pqv, stored with q fastest)
//
// which the fused B C/D kernel reads as its K-major P-side operand (K = q).  This is a
// memory-bound contraction (U in, A^T out, 2 x 4 N n^2 bytes per tau point, 4 n flops
// per byte) with a transposed, split output, so the kernel is built around its store:
//
//   * work items are (P, q block h, v block) with q blocks of 128 aligned to P, so the
//     output of an item is one dense box of A^T[P] (q contiguous) that TMA stores from
//     shared memory; the rows of a q block past n are the next P's (computed, never
//     stored: the store box is clipped at q = n);
//   * TMEM lane = q, column = v: an epilogue thread holds one q and 32 consecutive v of
//     a chunk, writes them as BF16 hi and lo into a [32 v][128 q] staging box (lanes
//     along q: conflict-free), and one thread per half of the columns issues the two
//     TMA stores (cp.async.bulk.tensor, bulk groups) of the chunk;
//   * two TMEM accumulators alternate between items, so the epilogue of one item runs
//     while the MMAs of the next accumulate.
//
// Warp roles as in split_gemm_kernel: warp 0 (one lane) loads the 64-deep K stages of
// U rows and G(-tau) rows (hi and lo, 128-byte swizzle; a last K block of at most 16 or
// 32 columns in boxes that narrow) by TMA; warp 1 allocates TMEM
// and one lane issues the 3 x 4 tcgen05.mma per stage (hi hi, hi lo, lo hi); warps 2-9
// drain, split and store.  Every wait is bounded in time (mbarriers, globaltimer); a
// wait that runs out sets *err and the CTA unwinds after draining its own copies, MMAs
// and bulk stores.
#pragma once

#include "tc_gemm.cuh"

namespace thc {
namespace tc {

struct SoxACfg {
  static constexpr int BV = 256;                           // v columns per item (TMEM columns per buffer)
  static constexpr int A_BYTES = BM * BKE * 2;             // 128 U rows x 64 s, BF16: 16 KB
  static constexpr int B_BYTES = BV * BKE * 2;             // up to 256 G rows x 64 s: 32 KB
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of both: 96 KB
  static constexpr int STAGES = 2;
  static constexpr int CHUNK = 32;                         // v columns per store box
  static constexpr int BOX = CHUNK * BM * 2;               // [32 v][128 q] BF16: 8 KB
  static constexpr int STAGING = 2 /*column halves*/ * 2 /*hi, lo*/ * BOX;
  static constexpr int SMEM = STAGES * STAGE + STAGING + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int TMEM_COLS = 2 * BV;
  static_assert(SMEM <= 232448, "shared memory per CTA");
};

struct SoxAArgs {
  int Pc;        // P in the block
  int n;         // AO count: q, v, s ranges
  int nh;        // q blocks per P: ceil(n / 128)
  int nvt;       // v blocks per item row: ceil(n / 256)
  int brows;     // rows of the G box: min(256, round-up-16(n))
  uint32_t tx;   // bytes per stage: 2 (128 + brows) 128
  int tail;      // 16 or 32: the last K block (n mod 64 <= tail) is loaded with boxes that wide; 0: 64
};

// U: rows P n + q of the block (K = s); G: rows v (K = s); At: 3-D (q, v, P) store maps;
// ut*, gt*: the narrow boxes of a shallow last K block.
struct SoxAMaps {
  CUtensorMap uh, ul, gh, gl, ath, atl, uth, utl, gth, gtl;
};

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the bulk stores of this thread have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the bulk stores of this thread are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the async (TMA) proxy
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(NTHREADS, 1)
    sox_a_kernel(const __grid_constant__ SoxAMaps maps, SoxAArgs a, int* err) {
  using C = SoxACfg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* staging = smem + C::STAGES * C::STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(staging + C::STAGING);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;  // [2] accumulator of an item complete
  uint64_t* acc_free = acc_full + 2;       // [2] accumulator drained
  uint64_t* written = acc_free + 2;        // [2] staging box of a column half filled (4 warps)
  uint64_t* freed = written + 2;           // [2] staging box of a column half read by its stores
  uint64_t* drain = freed + 2;             // every MMA of this CTA complete (unwind)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (a.n + BKE - 1) / BKE;
  const long long items = (long long)a.Pc * a.nh * a.nvt;
  // item i: v block fastest, then q block, then P
  auto decode = [&](long long i, int& P, int& h, int& vt) {
    vt = (int)(i % a.nvt);
    const long long r = i / a.nvt;
    h = (int)(r % a.nh);
    P = (int)(r / a.nh);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_free[i], NEPI);
      mbar_init(&written[i], 4);
      mbar_init(&freed[i], 1);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
    prefetch_map(&maps.uh);
    prefetch_map(&maps.ul);
    prefetch_map(&maps.gh);
    prefetch_map(&maps.gl);
    prefetch_map(&maps.ath);
    prefetch_map(&maps.atl);
    if (a.tail) {
      prefetch_map(&maps.uth);
      prefetch_map(&maps.utl);
      prefetch_map(&maps.gth);
      prefetch_map(&maps.gtl);
    }
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
      long long g = 0;  // running K-stage counter across items
      bool ok = true;
      for (long long i = blockIdx.x; i < items && ok; i += gridDim.x) {
        int P, h, vt;
        decode(i, P, h, vt);
        const int urow = P * a.n + h * BM, grow = vt * C::BV;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % C::STAGES);
          if (!mbar_wait(&empty[s], ((uint32_t)(g / C::STAGES) & 1) ^ 1)) {
            atomicExch(err, 21);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * C::STAGE;
          const bool tl = a.tail && kb == nkb - 1;  // narrow last K block: rows of 2 a.tail bytes
          mbar_arrive_expect_tx(&full[s], tl ? (uint32_t)(2 * (BM + a.brows) * 2 * a.tail) : a.tx);
          tma_load_3d(st, tl ? &maps.uth : &maps.uh, &full[s], kb * BKE, urow, 0);
          tma_load_3d(st + C::A_BYTES, tl ? &maps.utl : &maps.ul, &full[s], kb * BKE, urow, 0);
          tma_load_3d(st + 2 * C::A_BYTES, tl ? &maps.gth : &maps.gh, &full[s], kb * BKE, grow, 0);
          tma_load_3d(st + 2 * C::A_BYTES + C::B_BYTES, tl ? &maps.gtl : &maps.gl, &full[s], kb * BKE, grow, 0);
        }
      }
      if (!drain_stages(full, C::STAGES, g)) atomicExch(err, 24);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0, local = 0;
      bool ok = true;
      for (long long i = blockIdx.x; i < items && ok; i += gridDim.x, ++local) {
        int P, h, vt;
        decode(i, P, h, vt);
        const int width = min(C::BV, a.n - vt * C::BV);
        const uint32_t idesc = idesc_bf16(BM, (width + 15) & ~15);
        const int buf = (int)(local & 1);
        if (!mbar_wait(&acc_free[buf], ((uint32_t)(local >> 1) & 1) ^ 1)) {
          atomicExch(err, 22);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + static_cast<uint32_t>(buf * C::BV);
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % C::STAGES);
          if (!mbar_wait(&full[s], (uint32_t)(g / C::STAGES) & 1)) {
            atomicExch(err, 22);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * C::STAGE);
          const bool tl = a.tail && kb == nkb - 1;
          auto desc = [&](uint32_t addr) { return tl ? narrow_desc(addr, a.tail) : sw128_desc(addr); };
          const uint64_t ah = desc(base), al = desc(base + C::A_BYTES);
          const uint64_t bh = desc(base + 2 * C::A_BYTES), bl = desc(base + 2 * C::A_BYTES + C::B_BYTES);
          const int ksteps = min(BKE / 16, (a.n - kb * BKE + 15) >> 4);
#pragma unroll
          for (int k = 0; k < BKE / 16; ++k) {
            if (k < ksteps) {
              const uint64_t off = static_cast<uint64_t>((k * 32) >> 4);
              mma_bf16(d, ah + off, bh + off, idesc, (kb | k) != 0);
              mma_bf16(d, ah + off, bl + off, idesc, 1u);
              mma_bf16(d, al + off, bh + off, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
          if (kb == nkb - 1) mma_commit(&acc_full[buf]);
        }
      }
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicExch(err, 25);
    }
  } else {
    // warp (quarter, half): TMEM lanes 32 quarter .. (q rows), columns 128 half .. of the buffer
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int qloc = quarter * 32 + lane;
    __nv_bfloat16* box_hi = reinterpret_cast<__nv_bfloat16*>(staging + half * 2 * C::BOX);
    __nv_bfloat16* box_lo = reinterpret_cast<__nv_bfloat16*>(staging + half * 2 * C::BOX + C::BOX);
    const bool issuer = quarter == 0 && lane == 0;  // issues the stores of this column half
    long long local = 0, chunk = 0;                  // items and chunks of this half handled
    bool ok = true;
    for (long long i = blockIdx.x; i < items && ok; i += gridDim.x, ++local) {
      int P, h, vt;
      decode(i, P, h, vt);
      const int width = min(C::BV, a.n - vt * C::BV);
      const int buf = (int)(local & 1);
      if (!mbar_wait(&acc_full[buf], (uint32_t)(local >> 1) & 1)) {
        if (lane == 0) atomicExch(err, 23);
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t src = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + buf * C::BV + half * (C::BV / 2);
#pragma unroll 1
      for (int c = 0; c < C::BV / 2; c += C::CHUNK) {
        const int col = half * (C::BV / 2) + c;  // first v of the chunk within the item
        if (col >= width) break;                 // the same for all four warps of the half
        uint32_t r[32];
        tmem_ld16(src + c, r);
        tmem_ld16(src + c + 16, r + 16);
        tmem_wait_ld();
        // the staging box of this half is free once the previous chunk's stores have read it
        if (!mbar_wait(&freed[half], ((uint32_t)chunk & 1) ^ 1)) {
          if (lane == 0) atomicExch(err, 26);
          ok = false;
          break;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float x = __uint_as_float(r[j]);
          const __nv_bfloat16 hv = __float2bfloat16_rn(x);
          box_hi[j * BM + qloc] = hv;
          box_lo[j * BM + qloc] = __float2bfloat16_rn(x - __bfloat162float(hv));
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&written[half]);
        if (issuer) {
          if (!mbar_wait(&written[half], (uint32_t)chunk & 1)) {
            atomicExch(err, 27);
            ok = false;
          } else {
            // A^T[P][v][q] box (q from 128 h, v from vt 256 + col, one P); clipped at q, v = n
            tma_store_3d(&maps.ath, box_hi, h * BM, vt * C::BV + col, P);
            tma_store_3d(&maps.atl, box_lo, h * BM, vt * C::BV + col, P);
            bulk_commit();
            bulk_wait_read();
            mbar_arrive(&freed[half]);
          }
        }
        ++chunk;
        if (!ok) break;
      }
      // every column of the accumulator has been read (the loads above completed)
      tc_fence_before();
      mbar_arrive(&acc_free[buf]);
    }
    if (issuer) bulk_wait_all();
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
