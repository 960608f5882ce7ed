// Launch counter, optional per-kernel-class timing with CUDA events, and one NVTX
// range per launch named after its kernel class (free unless a profiler such as
// Nsight Systems or ncu with NVTX filtering is attached).
#include <nvtx3/nvToolsExt.h>

#include "thc_internal.cuh"

namespace thc {

const char* kernel_class_name(int k) {
  static const char* names[K_COUNT] = {"u_build",  "project",  "sox_A",        "sox_B",  "sox_CD", "polarisation",
                                       "direct_VPi", "direct_W", "back_transform", "energy", "split", "sox_BCD",
                                       "check", "screen"};
  return (k >= 0 && k < K_COUNT) ? names[k] : "";
}

static cudaEvent_t pool_get(thc_ctx* ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int prof_begin(thc_ctx* ctx, int kclass, double flops, ProfRec* rec) {
  rec->kclass = kclass;
  rec->flops = flops;
  rec->e0 = rec->e1 = nullptr;
  if (ctx->prof_on) {
    rec->e0 = pool_get(ctx);
    rec->e1 = pool_get(ctx);
    if (!rec->e0 || !rec->e1) return fail(ctx, THC_ECUDA, "cudaEventCreate failed");
    THC_TRY(check_cuda(ctx, cudaEventRecord(rec->e0, ctx->stream), "profiler event"));
  }
  nvtxRangePushA(kernel_class_name(kclass));  // popped by prof_end, which every caller reaches
  return THC_OK;
}

int prof_end(thc_ctx* ctx, ProfRec* rec, cudaError_t launch_status, const char* what) {
  nvtxRangePop();
  THC_TRY(check_cuda(ctx, launch_status, what));
  ctx->launch_count += 1;
  if (!ctx->prof_on) return THC_OK;
  THC_TRY(check_cuda(ctx, cudaEventRecord(rec->e1, ctx->stream), "profiler event"));
  ctx->prof_pending.push_back(*rec);
  if (ctx->prof_pending.size() >= 8192) return prof_flush(ctx);
  return THC_OK;
}

int prof_flush(thc_ctx* ctx) {
  if (ctx->prof_pending.empty()) return THC_OK;
  THC_TRY(check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "profiler sync"));
  for (ProfRec& r : ctx->prof_pending) {
    float ms = 0.f;
    THC_TRY(check_cuda(ctx, cudaEventElapsedTime(&ms, r.e0, r.e1), "profiler elapsed"));
    ProfStat& s = ctx->prof_stat[r.kclass];
    s.launches += 1;
    s.ms += ms;
    s.flops += r.flops;
    ctx->prof_pool.push_back(r.e0);
    ctx->prof_pool.push_back(r.e1);
  }
  ctx->prof_pending.clear();
  return THC_OK;
}

void prof_release(thc_ctx* ctx) {
  for (ProfRec& r : ctx->prof_pending) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  ctx->prof_pending.clear();
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  ctx->prof_pool.clear();
}

}  // namespace thc
