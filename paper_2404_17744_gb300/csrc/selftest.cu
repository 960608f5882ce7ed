// Self-test of the bounded waits of the tensor-core kernels (no counterpart in
// the paper: it checks this library's own failure handling).
//
// One CTA does what a producer and an MMA lane of split_gemm_kernel or
// sox_bcd_kernel do when a wait runs out: it holds TMEM and a bulk copy in
// flight, waits on an mbarrier that no thread ever completes until the limit
// passes, then unwinds the same way (waits, bounded, for its copy and for its
// tensor-core operations, frees TMEM, returns) and reports through the error
// word.  Nothing faults, traps or spins without a limit.
#include "tc_gemm.cuh"
#include "thc_internal.cuh"

namespace thc {
namespace {

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

// err bits: 1 the wait ran out (expected), 2 the copy did not land in time, 4 the
// tensor-core drain did not complete in time.
__global__ void __launch_bounds__(64, 1) wait_selftest_kernel(const uint4* __restrict__ src,
                                                              unsigned long long limit_ns, int* err) {
  __shared__ __align__(128) uint8_t buf[1024];
  __shared__ __align__(8) uint64_t bars[3];  // [0] never completed, [1] copy landed, [2] drain
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bars[i], 1);
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_slot, 32);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    tc::mbar_arrive_expect_tx(&bars[1], sizeof(buf));
    bulk_copy(buf, src, sizeof(buf), &bars[1]);
    if (!tc::mbar_wait(&bars[0], 0, limit_ns)) atomicOr(err, 1);  // nothing arrives on bars[0]
    if (!tc::mbar_wait(&bars[1], 0)) atomicOr(err, 2);             // unwind: the copy has landed
  }
  if (warp == 1 && lane == 0) {
    tc::mma_commit(&bars[2]);  // unwind: every tensor-core operation of this thread is complete
    if (!tc::mbar_wait(&bars[2], 0)) atomicOr(err, 4);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 32);
  }
}

}  // namespace
}  // namespace thc

extern "C" int thc_wait_selftest(long long limit_ns, void* stream) {
  using namespace thc;
  if (limit_ns < 1000 || limit_ns > 1000000000LL)
    return fail(nullptr, THC_EINVAL, "thc_wait_selftest: limit_ns must lie in [1e3, 1e9]");
  const cudaStream_t st = (cudaStream_t)stream;
  void* mem = nullptr;
  if (cudaMalloc(&mem, 2048) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, THC_ENOMEM, "thc_wait_selftest: cudaMalloc failed");
  }
  int flags = 0;
  int rc = check_cuda(nullptr, cudaMemsetAsync(mem, 0, 2048, st), "thc_wait_selftest: clear");
  if (rc == THC_OK) {
    wait_selftest_kernel<<<1, 64, 0, st>>>(static_cast<const uint4*>(mem), (unsigned long long)limit_ns,
                                           reinterpret_cast<int*>(static_cast<char*>(mem) + 1024));
    rc = check_cuda(nullptr, cudaGetLastError(), "thc_wait_selftest: launch");
  }
  if (rc == THC_OK)
    rc = check_cuda(nullptr, cudaMemcpyAsync(&flags, static_cast<char*>(mem) + 1024, sizeof(int),
                                             cudaMemcpyDeviceToHost, st), "thc_wait_selftest: read");
  if (rc == THC_OK) rc = check_cuda(nullptr, cudaStreamSynchronize(st), "thc_wait_selftest: sync");
  cudaFree(mem);
  if (rc != THC_OK) return rc;
  if (flags == 1) return fail(nullptr, THC_ETIMEOUT, "thc_wait_selftest: the wait ran out and the CTA unwound");
  return fail(nullptr, THC_ECUDA, "thc_wait_selftest: unexpected status " + std::to_string(flags));
}
