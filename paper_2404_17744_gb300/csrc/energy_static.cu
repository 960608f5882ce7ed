// Allocation-free variant of the Galitskii-Migdal energy reduction.
//
// thc_energy keeps its per-tau partial traces, the weights and the result in
// device memory that the context allocated.  Some callers cannot allocate
// device memory at all: code running under an external memory manager that
// owns every byte of the GPU, plugins that may only touch buffers handed to
// them, or a loop driver that must not call cudaMalloc after start-up.  For
// them thc_energy_static computes the same number with its scratch in the
// fixed array below, so it needs neither a context nor any allocation.
#include <mutex>
#include <string>

#include "thc_internal.cuh"

namespace {

constexpr int kMaxTau = THC_STATIC_MAX_TAU;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: [0, kMaxTau) partial traces,
// [kMaxTau, 2 kMaxTau) weights, [2 kMaxTau] the result.  65 KiB per device,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_energy_scratch[2 * kMaxTau + 32];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_energy_scratch on the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return thc::check_cuda(nullptr, e, "thc_energy_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return thc::fail(nullptr, THC_EINVAL, "thc_energy_static: device index above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess || !p) return thc::check_cuda(nullptr, e, "thc_energy_static: cudaGetSymbolAddress");
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return THC_OK;
}

// Partial traces t_k = sum_ij Gb_k[i, j] S_k[j, i], one CTA per tau point
// (same arithmetic and order as the context path).
__global__ void static_trace_kernel(int n, const double* __restrict__ Gb0, long long sGb,
                                    const double* __restrict__ S, double* __restrict__ part) {
  const long long k = blockIdx.x;
  const double* g = Gb0 + k * sGb;
  const double* s = S + k * (long long)n * n;
  double acc = 0.0;
  const long long nn = (long long)n * n;
  for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const long long i = idx / n, j = idx - i * n;
    acc = fma(g[idx], s[j * n + i], acc);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[k] = v;
  }
}

// E = -sum_k w_k t_k in a fixed order (one warp).
__global__ void static_sum_kernel(int n_tau, const double* __restrict__ part, const double* __restrict__ w,
                                  double* __restrict__ out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n_tau; k += 32) acc = fma(w[k], part[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) out[0] = -acc;
}

}  // namespace

extern "C" int thc_energy_static(int n_ao, int n_tau, const double* G_tau, const double* G_bmt,
                                 const double* Sigma_tau, const double* tau_weights, double* E_dyn, void* stream) {
  using namespace thc;
  if (n_ao < 1 || n_tau < 1) return fail(nullptr, THC_EINVAL, "thc_energy_static: need n_ao >= 1 and n_tau >= 1");
  if (n_tau > kMaxTau)
    return fail(nullptr, THC_EINVAL,
                "thc_energy_static: n_tau = " + std::to_string(n_tau) + " exceeds the static scratch limit of " +
                    std::to_string(kMaxTau) + " tau points; use thc_energy");
  if (!G_tau || !Sigma_tau || !tau_weights || !E_dyn)
    return fail(nullptr, THC_EINVAL, "thc_energy_static: NULL argument");
  double* scratch = nullptr;
  THC_TRY(scratch_address(&scratch));
  double* part = scratch;
  double* w = scratch + kMaxTau;
  double* out = scratch + 2 * kMaxTau;
  cudaStream_t s = (cudaStream_t)stream;
  const long long nn = (long long)n_ao * n_ao;
  const double* gb0 = G_bmt ? G_bmt : G_tau + (long long)(n_tau - 1) * nn;
  const long long sgb = G_bmt ? nn : -nn;
  // Every slot read below is written earlier in this call, so nothing left by
  // a previous call is used and nothing needs clearing.
  THC_TRY(check_cuda(nullptr, cudaMemcpyAsync(w, tau_weights, sizeof(double) * n_tau, cudaMemcpyHostToDevice, s),
                     "thc_energy_static: copy weights"));
  static_trace_kernel<<<(unsigned)n_tau, 256, 0, s>>>(n_ao, gb0, sgb, Sigma_tau, part);
  THC_TRY(check_cuda(nullptr, cudaGetLastError(), "thc_energy_static: trace"));
  static_sum_kernel<<<1, 32, 0, s>>>(n_tau, part, w, out);
  THC_TRY(check_cuda(nullptr, cudaGetLastError(), "thc_energy_static: sum"));
  THC_TRY(check_cuda(nullptr, cudaMemcpyAsync(E_dyn, out, sizeof(double), cudaMemcpyDeviceToHost, s),
                     "thc_energy_static: copy energy"));
  return check_cuda(nullptr, cudaStreamSynchronize(s), "thc_energy_static: sync");
}
