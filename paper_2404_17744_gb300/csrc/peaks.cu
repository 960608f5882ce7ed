// FP64 peak of the device, measured: the denominator of the FP64 path's roofline.
//
// GB300 has no FP64 tensor-core kind, so every FP64 contraction here runs on the
// DFMA pipe; its peak is the rate of independent fused multiply-adds.  The kernel
// below keeps 8 independent FMA chains per thread (enough to cover the DFMA
// latency) in 4 resident CTAs of 256 threads per SM, and every chain depends only
// on its own previous value, so nothing but the DFMA issue rate limits it.
#include <cuda_runtime.h>

#include "thc_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) dfma_rate_kernel(long long iters, double b, double c, double* out) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1.0 + 1e-9 * (threadIdx.x + 8 * i);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 12345.678) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" int thc_fp64_dfma_rate(long long iters, double* tflops, double* ms, void* stream) {
  using namespace thc;
  if (iters < 1 || iters > (1LL << 40) || !tflops)
    return fail(nullptr, THC_EINVAL, "thc_fp64_dfma_rate: need 1 <= iters <= 2^40 and a non-NULL output");
  const cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  THC_TRY(check_cuda(nullptr, cudaGetDevice(&dev), "thc_fp64_dfma_rate: device"));
  THC_TRY(check_cuda(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                     "thc_fp64_dfma_rate: SM count"));
  const int blocks = 4 * sms;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, THC_ENOMEM, "thc_fp64_dfma_rate: cudaMalloc failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = check_cuda(nullptr, cudaEventCreate(&e0), "thc_fp64_dfma_rate: event");
  if (rc == THC_OK) rc = check_cuda(nullptr, cudaEventCreate(&e1), "thc_fp64_dfma_rate: event");
  float t = 0.f;
  if (rc == THC_OK) {
    dfma_rate_kernel<<<blocks, 256, 0, st>>>(iters / 8 + 1, 0.999999, 1e-7, out);  // warm-up
    cudaEventRecord(e0, st);
    dfma_rate_kernel<<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, out);
    cudaEventRecord(e1, st);
    rc = check_cuda(nullptr, cudaGetLastError(), "thc_fp64_dfma_rate: launch");
  }
  if (rc == THC_OK) rc = check_cuda(nullptr, cudaEventSynchronize(e1), "thc_fp64_dfma_rate: sync");
  if (rc == THC_OK) rc = check_cuda(nullptr, cudaEventElapsedTime(&t, e0, e1), "thc_fp64_dfma_rate: time");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != THC_OK) return rc;
  const double flops = 2.0 * 8.0 * (double)iters * 256.0 * blocks;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return THC_OK;
}
