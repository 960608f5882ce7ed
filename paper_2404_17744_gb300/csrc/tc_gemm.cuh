// Split-precision contraction on the 5th-generation tensor cores (sm_103a).
//
//   C[b][m][n] = sum_k A[b][m][k] B[b][n][k]
//             ~= sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)       (FP32 accumulation in TMEM)
//
// with every FP64 operand x stored as a pair of BF16 values hi = bf16(x),
// lo = bf16(x - hi) (about 17 significant bits together).  The constant
// operands X and V may carry a third term lo2 = bf16(x - hi - lo) (AT = 3,
// one more product Alo2 Bhi per step): their rounding is coherent across the
// whole scheme and otherwise dominates the error of the energy.  A data operand may
// carry the third term as well (BT = 3, with AT = 3: two more products, hi lo2 and
// lo lo, so that every product down to 2^-16 relative is kept).  Both operands are
// K-major (k contiguous), which every contraction of the THC scheme can be
// brought to by the symmetry of G, U_Pqs and V or by writing its producer's
// output transposed.
//
// The kernel is persistent: one CTA per SM walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... of all batches (tile order: row block fastest,
// so consecutive tiles share their B operand), and every role counts K stages
// with one running counter across tiles.  The producer therefore loads the
// next tile while the current one drains and stores, and the MMA warp runs
// ahead into the two TMEM stage buffers during the store phase.
// Each tile is 128 x BN, computed by three warp roles:
//   warp 0    one lane issues the TMA loads (128-byte swizzle) of the four
//             (AT = 3: five) operand tiles of each 64-deep K stage into a
//             STAGES-deep ring;
//   warp 1    allocates TMEM; one lane issues the (AT + 1 + 2 (BT - 2)) x 4 tcgen05.mma
//             (kind::f16, M = 128, N = BN, K = 16) of a stage into one of two
//             TMEM accumulators (stages alternate between them) and commits
//             the stage back to the producer and to the epilogue (ragged
//             edges: the last K stage issues only the steps that reach below
//             K, and the last column tile uses N = round-up-16 of its width);
//   warps 2-9 drain each finished stage accumulator with tcgen05.ld into FP32
//             registers (warp w owns TMEM lanes 32 (w % 4) .. and one half of
//             the columns), free it for the stage after next, and finally hand
//             32 x 32 chunks, staged in a private XOR-swizzled shared-memory
//             tile, to the epilogue functor, which the whole warp runs with
//             coalesced global accesses.
// Draining every stage ("promotion") keeps the tensor core's internal
// accumulation to one 64-deep stage.  Measured on GB300 with exactly
// representable products, the FP32 accumulator is rounded toward zero after
// every MMA instruction: sums of one sign lose about a quarter ulp per
// instruction, a bias that grows with the number of instructions accumulated in
// TMEM (-2.7e-7 relative at K = 200 in one chunk, -7.7e-8 for 64-deep stages
// added in FP32 registers) and that the chained contractions of the direct term
// carry into the energy.  The promoted mode therefore also keeps the hi*hi
// products and the 2^-8 smaller correction products in separate TMEM
// accumulators (their truncation then scales with their own magnitude), and it
// runs every contraction with the three-term operands X and V (K from n to N).
// The remaining contractions (the SOX A step) run in the single-chunk mode
// (MULTI = false): the whole K accumulates in one TMEM buffer, tiles alternate
// between the two buffers (the epilogue of one tile overlaps the MMAs of the
// next), and the epilogue streams 32-column slices straight from TMEM without a
// register accumulator.
// Every mbarrier wait is bounded in time (globaltimer); a wait that runs out
// sets *err and the CTA unwinds: the producer waits (bounded) for every TMA
// stage it issued, the MMA lane commits its outstanding MMAs to a drain
// barrier and waits for it (bounded), and only then is TMEM freed and the CTA
// returns, so no copy or MMA lands in shared memory or TMEM that was given up.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace thc {
namespace tc {

constexpr int BM = 128;        // rows of a tile (TMEM lanes)
constexpr int BKE = 64;        // K elements per stage: one 128-byte swizzle row of BF16
constexpr int NTHREADS = 320;  // 10 warps: TMA, MMA, 8 epilogue
constexpr int NEPI = 256;      // epilogue threads
constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // 4 s per wait

// AT = number of BF16 terms of the A operand: 2 (hi, lo) or 3 (hi, lo, lo2 =
// bf16(x - hi - lo), about 24 significant bits together, for the constant
// operands X and V whose rounding otherwise dominates the energy error).
// BT = number of BF16 terms of the B operand: 2, or 3 for data operands kept to about
// 24 bits (then the products down to 2^-16 relative are all issued: hi hi, hi lo,
// lo hi, lo2 hi, hi lo2 and lo lo).
template <int BN, int AT = 2, int BT = 2>
struct Cfg {
  static constexpr int A_BYTES = BM * BKE * 2;
  static constexpr int B_BYTES = BN * BKE * 2;
  static constexpr int STAGE = AT * A_BYTES + BT * B_BYTES;
  static constexpr int TMEM_COLS = 2 * BN;   // two accumulators; BN in {128, 256}
  // promoted mode: each of the two stage buffers holds the hi*hi products and, in a second
  // accumulator, the small correction products (BN = 128 only)
  static constexpr int TMEM_COLS_MULTI = 4 * BN;
  static constexpr int HALF = BN / 2;         // columns per epilogue thread
  static constexpr int STAGING = 8 * 32 * 32 * 4;  // one swizzled 32 x 32 FP32 tile per warp
  static constexpr int FIXED = STAGING + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int STAGES = ((232448 - FIXED) / STAGE) >= 3 ? 3 : 2;
  static constexpr int SMEM = STAGES * STAGE + FIXED;
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(BN == 128 || BN == 256, "tile width");
  static_assert(AT == 2 || AT == 3, "A operand terms");
  static_assert(BT == 2 || (BT == 3 && AT == 3), "B operand terms (three only with a three-term A)");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Waits until the phase of parity `parity` of *bar has completed; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
  const uint32_t addr = smem_u32(bar);
  const unsigned long long t0 = globaltimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

// Unwind of a producer: waits (bounded) for the last phase armed on each of the
// `stages` full barriers, i.e. for every TMA copy this thread issued.  `issued` is the
// number of stage uses armed so far (stage g % stages, phase g / stages).
__device__ __forceinline__ bool drain_stages(uint64_t* full, int stages, long long issued) {
  bool ok = true;
  for (int s = 0; s < stages; ++s) {
    // last use g of stage s below `issued`: g = s + stages * j with the largest j
    if (issued <= s) continue;
    const long long last = s + (long long)stages * ((issued - 1 - s) / stages);
    ok &= mbar_wait(&full[s], (uint32_t)(last / stages) & 1);
  }
  return ok;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;            // leading byte offset (unused for swizzled K-major)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;    // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;            // version
  d |= static_cast<uint64_t>(2) << 61;            // SWIZZLE_128B
  return d;
}

// The same for a narrow K block of 16 or 32 BF16 per row (32- or 64-byte rows, 32- or
// 64-byte swizzle, 8-row groups 256 or 512 bytes apart): the last K block of a contraction
// whose depth leaves only that much, loaded with a box as narrow.
__device__ __forceinline__ uint64_t narrow_desc(uint32_t saddr, int width) {
  const uint64_t row = static_cast<uint64_t>(width) * 2;  // bytes per row
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= ((8 * row) >> 4) << 32;                             // stride byte offset: one 8-row group
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(width == 16 ? 6 : 4) << 61;   // SWIZZLE_32B or SWIZZLE_64B
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns into r[0..15] (no wait):
// thread t reads lane (base + t).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 TMEM lanes x 16 consecutive 32-bit columns, added into acc[0..15]:
// thread t reads lane (base + t).
__device__ __forceinline__ void tmem_ld16_add(uint32_t taddr, float* acc) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] += __uint_as_float(r[i]);
}

// A 32 x 32 FP32 tile with XOR swizzle: element (r, c) at r * 32 + (c ^ r), so
// that both row walks (fixed r) and column walks (fixed c) are bank-conflict free.
struct TileRef {
  float* p;
  __device__ __forceinline__ float& operator()(int r, int c) const { return p[r * 32 + (c ^ r)]; }
};

// Operand maps: each is a 3-D tensor map (k, row, batch) over BF16 with a
// 64 x rows box and 128-byte swizzle.  batched = 0 pins the batch coordinate to 0.
struct Operands {
  int a_batched, b_batched;
};

template <int BN, bool MULTI, int AT, class Epi, int BT = 2>
__global__ void __launch_bounds__(NTHREADS, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                      const __grid_constant__ CUtensorMap mAlo2, const __grid_constant__ CUtensorMap mBhi,
                      const __grid_constant__ CUtensorMap mBlo, const __grid_constant__ CUtensorMap mBlo2, int M, int N,
                      int K, int batch, Operands ops, Epi epi, int* err) {
  using C = Cfg<BN, AT, BT>;
  constexpr int B_OFF = AT * C::A_BYTES;  // B hi, then B lo, after the A terms of a stage
  constexpr int TCOLS = MULTI ? C::TMEM_COLS_MULTI : C::TMEM_COLS;
  static_assert(TCOLS <= 512, "TMEM columns");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* staging = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE + C::STAGING);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;  // [2] stage accumulator ready for the epilogue
  uint64_t* acc_free = acc_full + 2;       // [2] stage accumulator drained
  uint64_t* drain = acc_free + 2;          // every MMA of this CTA complete (unwind)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (K + BKE - 1) / BKE;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const long long tiles = (long long)tm * tn * batch;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_free[i], NEPI);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
    prefetch_map(&mAhi);
    prefetch_map(&mAlo);
    if (AT == 3) prefetch_map(&mAlo2);
    if (BT == 3) prefetch_map(&mBlo2);
    prefetch_map(&mBhi);
    prefetch_map(&mBlo);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;  // running K-stage counter across tiles
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int mt = (int)(t % tm), nt = (int)((t / tm) % tn), b = (int)(t / ((long long)tm * tn));
        const int ab = ops.a_batched ? b : 0, bb = ops.b_batched ? b : 0;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % C::STAGES);
          const uint32_t r = (uint32_t)(g / C::STAGES);
          if (!mbar_wait(&empty[s], (r & 1) ^ 1)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * C::STAGE;
          mbar_arrive_expect_tx(&full[s], C::STAGE);
          tma_load_3d(st, &mAhi, &full[s], kb * BKE, mt * BM, ab);
          tma_load_3d(st + C::A_BYTES, &mAlo, &full[s], kb * BKE, mt * BM, ab);
          if (AT == 3) tma_load_3d(st + 2 * C::A_BYTES, &mAlo2, &full[s], kb * BKE, mt * BM, ab);
          tma_load_3d(st + B_OFF, &mBhi, &full[s], kb * BKE, nt * BN, bb);
          tma_load_3d(st + B_OFF + C::B_BYTES, &mBlo, &full[s], kb * BKE, nt * BN, bb);
          if (BT == 3) tma_load_3d(st + B_OFF + 2 * C::B_BYTES, &mBlo2, &full[s], kb * BKE, nt * BN, bb);
        }
      }
      // every copy issued has landed before the CTA may leave (immediate unless a wait ran out)
      if (!drain_stages(full, C::STAGES, g)) atomicExch(err, 4);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0, local = 0;  // K stages and tiles handled by this CTA
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++local) {
        // a ragged last column tile multiplies only its round-up-to-16 width (columns beyond
        // it stay unwritten in TMEM; every epilogue skips columns >= N)
        const int nt = (int)((t / tm) % tn);
        const int n_eff = min(BN, (N - nt * BN + 15) & ~15);
        const uint32_t idesc = idesc_bf16(BM, n_eff);
        if (!MULTI) {  // one accumulator per tile, alternating between the two buffers
          const int buf = (int)(local & 1);
          if (!mbar_wait(&acc_free[buf], ((uint32_t)(local >> 1) & 1) ^ 1)) {
            atomicExch(err, 2);
            break;
          }
        }
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % C::STAGES);
          const int buf = MULTI ? (int)(g & 1) : (int)(local & 1);
          const uint32_t r = (uint32_t)(g / C::STAGES), use = (uint32_t)(g >> 1);
          if ((MULTI && !mbar_wait(&acc_free[buf], (use & 1) ^ 1)) || !mbar_wait(&full[s], r & 1)) {
            atomicExch(err, 2);
            ok = false;
            break;
          }
          tc_fence_after();
          // single-chunk: one accumulator per buffer; promoted: hi*hi into d, corrections into dc
          const uint32_t d = tmem + static_cast<uint32_t>(buf * (MULTI ? 2 * BN : BN));
          const uint32_t dc = MULTI ? d + BN : d;
          const uint32_t base = smem_u32(smem + s * C::STAGE);
          const uint64_t ah = sw128_desc(base), al = sw128_desc(base + C::A_BYTES);
          const uint64_t al2 = sw128_desc(base + 2 * C::A_BYTES);
          const uint64_t bh = sw128_desc(base + B_OFF), bl = sw128_desc(base + B_OFF + C::B_BYTES);
          const uint64_t bl2 = sw128_desc(base + B_OFF + 2 * C::B_BYTES);
          // the last stage of a ragged K issues only the 16-deep steps that reach below K
          const int ksteps = min(BKE / 16, (K - kb * BKE + 15) >> 4);
#pragma unroll
          for (int k = 0; k < BKE / 16; ++k) {
            if (k < ksteps) {
              const uint64_t off = static_cast<uint64_t>((k * 32) >> 4);  // 16 BF16 = 32 bytes along K
              mma_bf16(d, ah + off, bh + off, idesc, (MULTI ? k : (kb | k)) != 0);
              mma_bf16(dc, ah + off, bl + off, idesc, MULTI ? (k != 0) : 1u);
              mma_bf16(dc, al + off, bh + off, idesc, 1u);
              if (AT == 3) mma_bf16(dc, al2 + off, bh + off, idesc, 1u);
              if (BT == 3) {
                mma_bf16(dc, ah + off, bl2 + off, idesc, 1u);
                mma_bf16(dc, al + off, bl + off, idesc, 1u);
              }
            }
          }
          mma_commit(&empty[s]);  // frees the smem stage once these MMAs have read it
          if (MULTI || kb == nkb - 1) mma_commit(&acc_full[buf]);  // accumulator ready
        }
      }
      // every MMA issued has completed before TMEM is freed (immediate unless a wait ran out)
      mma_commit(drain);
      if (!mbar_wait(drain, 0)) atomicExch(err, 5);
    }
  } else if (!MULTI) {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const TileRef tile{staging + (warp - 2) * 32 * 32};
    long long local = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
      const int mt = (int)(t % tm), nt = (int)((t / tm) % tn), b = (int)(t / ((long long)tm * tn));
      const int m0 = mt * BM, n0 = nt * BN, buf = (int)(local & 1);
      if (!mbar_wait(&acc_full[buf], (uint32_t)(local >> 1) & 1)) {
        if (lane == 0) atomicExch(err, 3);
        break;
      }
      tc_fence_after();
      const uint32_t src = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + buf * BN + half * C::HALF;
      const int row0 = m0 + quarter * 32;
#pragma unroll 1
      for (int c = 0; c < C::HALF; c += 32) {
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
        tmem_ld16_add(src + c, v);
        tmem_ld16_add(src + c + 16, v + 16);
#pragma unroll
        for (int j = 0; j < 32; ++j) tile(lane, j) = v[j];
        __syncwarp();
        const int col0 = n0 + half * C::HALF + c;
        if (col0 < N) epi(b, row0, col0, tile, lane, M, N);
        __syncwarp();
      }
      tc_fence_before();
      mbar_arrive(&acc_free[buf]);
    }
  } else {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + half * C::HALF;
    const TileRef tile{staging + (warp - 2) * 32 * 32};
    long long g = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int mt = (int)(t % tm), nt = (int)((t / tm) % tn), b = (int)(t / ((long long)tm * tn));
      const int m0 = mt * BM, n0 = nt * BN;
      float acc[C::HALF];
#pragma unroll
      for (int i = 0; i < C::HALF; ++i) acc[i] = 0.f;
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int buf = (int)(g & 1);
        const uint32_t use = (uint32_t)(g >> 1);
        if (!mbar_wait(&acc_full[buf], use & 1)) {
          if (lane == 0) atomicExch(err, 3);
          ok = false;
          break;
        }
        tc_fence_after();
        // the stage's hi*hi sum and its correction sum, 32 columns of each at a time
#pragma unroll
        for (int c0 = 0; c0 < C::HALF; c0 += 32) {
          uint32_t r[32], q[32];
          const uint32_t src = lane_base + buf * 2 * BN + c0;
          tmem_ld16(src, r);
          tmem_ld16(src + 16, r + 16);
          tmem_ld16(src + BN, q);
          tmem_ld16(src + BN + 16, q + 16);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i) acc[c0 + i] += __uint_as_float(r[i]) + __uint_as_float(q[i]);
        }
        tc_fence_before();
        mbar_arrive(&acc_free[buf]);
      }
      if (!ok) break;
      __syncwarp();
      const int row0 = m0 + quarter * 32;
#pragma unroll
      for (int c = 0; c < C::HALF; c += 32) {
        const int col0 = n0 + half * C::HALF + c;
#pragma unroll
        for (int j = 0; j < 32; ++j) tile(lane, j) = acc[c + j];
        __syncwarp();
        if (col0 < N) epi(b, row0, col0, tile, lane, M, N);
        __syncwarp();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TCOLS);
  }
}

}  // namespace tc
}  // namespace thc
