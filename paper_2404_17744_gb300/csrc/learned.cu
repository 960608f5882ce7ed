// Learned self-energy proposals for the self-consistency loop (no counterpart
// in the paper; it accelerates the loop the paper iterates to convergence,
// Sec. II.A, and never changes its fixed point: every proposal is an input
// self-energy that the exact Sigma evaluation of the next iteration judges).
//
// A two-layer perceptron, shared by all matrix elements e of Sigma, maps the
// IR coefficients of one element and their last change,
//     x_e = [ c_k[:, e] / s_c ,  (c_k - c_{k-1})[:, e] / s_d ]        (2 L inputs)
// through a ReLU layer of H units to a correction of its coefficients,
//     c_prop[:, e] = c_k[:, e] + s_d * MLP(x_e)                        (L outputs).
// It is trained on a loop's own trajectory: samples (j, e) with input x built
// from c_j, c_{j-1} and target (c_latest - c_j) / s_d(j), where s_c is the
// RMS of the latest iterate and s_d(j) the RMS of the change c_j - c_{j-1}.
// Weights are FP16 in the forward and backward passes with FP32 master
// copies, FP32 accumulation and Adam; every contraction runs in the FP32
// SIMT tile below.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "dfma_tile.cuh"
#include "thc_internal.cuh"
#include "thc_learned.h"

namespace {

// ----------------------------------------------------------- FP32 tile GEMM
// C(m, n) = sum_k A(m, k) B(k, n) with A(m, k) = A[m ra + k ca], B(k, n) = B[k rb + n cb]
// (float or half operands), epilogue epi(m, n, acc).  64 x 64 x 16 tiles, 256 threads.
template <class T>
__device__ __forceinline__ float ld(const T* p, long long i);
template <>
__device__ __forceinline__ float ld<float>(const float* p, long long i) { return p[i]; }
template <>
__device__ __forceinline__ float ld<__half>(const __half* p, long long i) { return __half2float(p[i]); }

template <class TA, class TB, class Epi>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const TA* __restrict__ A, long long ra,
                                                    long long ca, const TB* __restrict__ B, long long rb, long long cb,
                                                    Epi epi) {
  __shared__ float As[16][65], Bs[16][65];
  const int t = threadIdx.x, tm = t >> 4, tn = t & 15;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = t; i < 16 * 64; i += 256) {
      const int kk = i >> 6, mm = i & 63;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? ld(A, (long long)m * ra + (long long)k * ca) : 0.f;
      const int n = n0 + mm;
      Bs[kk][mm] = (n < N && k < K) ? ld(B, (long long)k * rb + (long long)n * cb) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + tm * 4 + i, n = n0 + tn * 4 + j;
      if (m < M && n < N) epi(m, n, acc[i][j]);
    }
}

template <class TA, class TB, class Epi>
cudaError_t sgemm(cudaStream_t s, int M, int N, int K, const TA* A, long long ra, long long ca, const TB* B,
                  long long rb, long long cb, const Epi& e) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  sgemm_kernel<<<dim3((M + 63) / 64, (N + 63) / 64), 256, 0, s>>>(M, N, K, A, ra, ca, B, rb, cb, e);
  return cudaGetLastError();
}

// Z1 = acc + b1; A1 = relu(Z1)
struct EpiHidden {
  float *Z, *A;
  const float* b;
  int H;
  __device__ void operator()(int m, int n, float v) const {
    const float z = v + b[n];
    Z[(long long)m * H + n] = z;
    A[(long long)m * H + n] = z > 0.f ? z : 0.f;
  }
};
// Y = acc + b2
struct EpiOut {
  float* Y;
  const float* b;
  int D;
  __device__ void operator()(int m, int n, float v) const { Y[(long long)m * D + n] = v + b[n]; }
};
// plain store
struct EpiStore {
  float* C;
  int ld;
  __device__ void operator()(int m, int n, float v) const { C[(long long)m * ld + n] = v; }
};
// dZ1 = acc * (Z1 > 0)
struct EpiReluGrad {
  float* dZ;
  const float* Z;
  int H;
  __device__ void operator()(int m, int n, float v) const {
    const long long o = (long long)m * H + n;
    dZ[o] = Z[o] > 0.f ? v : 0.f;
  }
};

// dY = 2 (Y - T) / (B D); part[b] = sum_o (Y - T)^2 for the loss
__global__ void out_grad_kernel(int B, int D, const float* __restrict__ Y, const float* __restrict__ T,
                                float* __restrict__ dY, float* __restrict__ part) {
  const int b = blockIdx.x * blockDim.y + threadIdx.y;
  if (b >= B) return;
  float acc = 0.f;
  const float sc = 2.f / ((float)B * (float)D);
  for (int o = threadIdx.x; o < D; o += 32) {
    const long long i = (long long)b * D + o;
    const float r = Y[i] - T[i];
    dY[i] = sc * r;
    acc = fmaf(r, r, acc);
  }
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (threadIdx.x == 0) part[b] = acc;
}

// column sums: out[c] = sum_r X[r][c] (fixed order per column)
__global__ void colsum_kernel(int R, int C, const float* __restrict__ X, float* __restrict__ out) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (int r = threadIdx.x; r < R; r += blockDim.x) acc += X[(long long)r * C + c];
  __shared__ float red[32];
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if (threadIdx.x == 0) out[c] = acc;
  }
}

// Adam on FP32 master weights; refreshes the FP16 working copy when h != null.
__global__ void adam_kernel(long long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __half* __restrict__ h, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (h) h[i] = __float2half_rn(wi);
  }
}

__global__ void to_half_kernel(long long n, const float* __restrict__ w, __half* __restrict__ h) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    h[i] = __float2half_rn(w[i]);
}

__global__ void sum_f_kernel(int n, const float* __restrict__ p, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) acc += p[i];
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (threadIdx.x == 0) out[0] = acc;
}

int blocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

// ====================================================================== MLP
struct thc_mlp {
  int din = 0, H = 0, dout = 0, max_batch = 0;
  cudaStream_t stream = nullptr;
  long long t = 0;  // Adam step
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;       // FP32 master
  __half *W1h = nullptr, *W2h = nullptr;                                  // FP16 working copies
  float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr;   // gradients
  float *mW1 = nullptr, *vW1 = nullptr, *mb1 = nullptr, *vb1 = nullptr;   // Adam moments
  float *mW2 = nullptr, *vW2 = nullptr, *mb2 = nullptr, *vb2 = nullptr;
  float *Z1 = nullptr, *A1 = nullptr, *Y = nullptr, *dY = nullptr, *dZ1 = nullptr, *part = nullptr;
  double* loss = nullptr;
  std::vector<void*> owned;
  std::string err;
};

namespace {

int mfail(thc_mlp* m, int code, const std::string& msg) {
  if (m) m->err = msg;
  return thc::fail(nullptr, code, msg);
}
int mcheck(thc_mlp* m, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return THC_OK;
  return mfail(m, e == cudaErrorMemoryAllocation ? THC_ENOMEM : THC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
template <class T>
int malloc_m(thc_mlp* m, T** p, size_t n, const char* what) {
  *p = nullptr;
  if (cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return mfail(m, THC_ENOMEM, std::string("cudaMalloc ") + what);
  }
  m->owned.push_back(*p);
  return THC_OK;
}

// forward on X (B x din) -> m->Y (B x dout); keeps Z1, A1 for the backward pass
int mlp_forward(thc_mlp* m, int B, const float* X) {
  const cudaStream_t s = m->stream;
  THC_TRY(mcheck(m, sgemm(s, B, m->H, m->din, X, m->din, 1, m->W1h, 1, m->din, EpiHidden{m->Z1, m->A1, m->b1, m->H}),
                 "mlp layer 1"));
  return mcheck(m, sgemm(s, B, m->dout, m->H, m->A1, m->H, 1, m->W2h, 1, m->H, EpiOut{m->Y, m->b2, m->dout}),
                "mlp layer 2");
}

// loss and gradients for targets T (B x dout) after mlp_forward
int mlp_backward(thc_mlp* m, int B, const float* X, const float* T) {
  const cudaStream_t s = m->stream;
  out_grad_kernel<<<(B + 7) / 8, dim3(32, 8), 0, s>>>(B, m->dout, m->Y, T, m->dY, m->part);
  THC_TRY(mcheck(m, cudaGetLastError(), "mlp output gradient"));
  sum_f_kernel<<<1, 32, 0, s>>>(B, m->part, m->loss);
  THC_TRY(mcheck(m, cudaGetLastError(), "mlp loss"));
  // dW2 = dY^T A1 ; db2 = colsum dY
  THC_TRY(mcheck(m, sgemm(s, m->dout, m->H, B, m->dY, 1, m->dout, m->A1, m->H, 1, EpiStore{m->gW2, m->H}), "dW2"));
  colsum_kernel<<<m->dout, 256, 0, s>>>(B, m->dout, m->dY, m->gb2);
  THC_TRY(mcheck(m, cudaGetLastError(), "db2"));
  // dZ1 = (dY W2) o [Z1 > 0] ; dW1 = dZ1^T X ; db1 = colsum dZ1
  THC_TRY(mcheck(m, sgemm(s, B, m->H, m->dout, m->dY, m->dout, 1, m->W2h, m->H, 1, EpiReluGrad{m->dZ1, m->Z1, m->H}),
                 "dZ1"));
  THC_TRY(mcheck(m, sgemm(s, m->H, m->din, B, m->dZ1, 1, m->H, X, m->din, 1, EpiStore{m->gW1, m->din}), "dW1"));
  colsum_kernel<<<m->H, 256, 0, s>>>(B, m->H, m->dZ1, m->gb1);
  return mcheck(m, cudaGetLastError(), "db1");
}

int mlp_adam(thc_mlp* m, float lr) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m->t += 1;
  const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
  const cudaStream_t s = m->stream;
  const long long n1 = (long long)m->H * m->din, n2 = (long long)m->dout * m->H;
  adam_kernel<<<blocks(n1), 256, 0, s>>>(n1, m->W1, m->gW1, m->mW1, m->vW1, m->W1h, lr, b1, b2, eps, c1, c2);
  adam_kernel<<<blocks(m->H), 256, 0, s>>>(m->H, m->b1, m->gb1, m->mb1, m->vb1, nullptr, lr, b1, b2, eps, c1, c2);
  adam_kernel<<<blocks(n2), 256, 0, s>>>(n2, m->W2, m->gW2, m->mW2, m->vW2, m->W2h, lr, b1, b2, eps, c1, c2);
  adam_kernel<<<blocks(m->dout), 256, 0, s>>>(m->dout, m->b2, m->gb2, m->mb2, m->vb2, nullptr, lr, b1, b2, eps, c1, c2);
  return mcheck(m, cudaGetLastError(), "adam");
}

}  // namespace

extern "C" {

int thc_mlp_init(thc_mlp** out, int d_in, int hidden, int d_out, int max_batch, const float* W1, const float* b1,
                 const float* W2, const float* b2, void* stream) {
  if (!out) return thc::fail(nullptr, THC_EINVAL, "thc_mlp_init: NULL out-pointer");
  *out = nullptr;
  if (d_in < 1 || hidden < 1 || d_out < 1 || max_batch < 1 || !W1 || !b1 || !W2 || !b2)
    return thc::fail(nullptr, THC_EINVAL, "thc_mlp_init: bad sizes or NULL weights");
  thc_mlp* m = new (std::nothrow) thc_mlp();
  if (!m) return thc::fail(nullptr, THC_ENOMEM, "thc_mlp_init: host allocation");
  m->din = d_in, m->H = hidden, m->dout = d_out, m->max_batch = max_batch;
  m->stream = (cudaStream_t)stream;
  const size_t n1 = (size_t)hidden * d_in, n2 = (size_t)d_out * hidden, B = max_batch;
  int rc = THC_OK;
  auto F = [&](float** p, size_t n, const char* w) { if (rc == THC_OK) rc = malloc_m(m, p, n, w); };
  F(&m->W1, n1, "W1"); F(&m->b1, hidden, "b1"); F(&m->W2, n2, "W2"); F(&m->b2, d_out, "b2");
  F(&m->gW1, n1, "gW1"); F(&m->gb1, hidden, "gb1"); F(&m->gW2, n2, "gW2"); F(&m->gb2, d_out, "gb2");
  F(&m->mW1, n1, "mW1"); F(&m->vW1, n1, "vW1"); F(&m->mb1, hidden, "mb1"); F(&m->vb1, hidden, "vb1");
  F(&m->mW2, n2, "mW2"); F(&m->vW2, n2, "vW2"); F(&m->mb2, d_out, "mb2"); F(&m->vb2, d_out, "vb2");
  F(&m->Z1, B * hidden, "Z1"); F(&m->A1, B * hidden, "A1"); F(&m->Y, B * d_out, "Y"); F(&m->dY, B * d_out, "dY");
  F(&m->dZ1, B * hidden, "dZ1"); F(&m->part, B, "loss partials");
  if (rc == THC_OK) rc = malloc_m(m, &m->W1h, n1, "W1 half");
  if (rc == THC_OK) rc = malloc_m(m, &m->W2h, n2, "W2 half");
  if (rc == THC_OK) rc = malloc_m(m, &m->loss, 1, "loss");
  const cudaStream_t s = m->stream;
  auto up = [&](float* d, const float* h, size_t n) {
    if (rc == THC_OK) rc = mcheck(m, cudaMemcpyAsync(d, h, 4 * n, cudaMemcpyDefault, s), "copy weights");
  };
  up(m->W1, W1, n1); up(m->b1, b1, hidden); up(m->W2, W2, n2); up(m->b2, b2, d_out);
  for (float* z : {m->mW1, m->vW1, m->mb1, m->vb1, m->mW2, m->vW2, m->mb2, m->vb2}) {
    const size_t n = (z == m->mW1 || z == m->vW1) ? n1 : (z == m->mW2 || z == m->vW2) ? n2
                     : (z == m->mb1 || z == m->vb1) ? (size_t)hidden : (size_t)d_out;
    if (rc == THC_OK) rc = mcheck(m, cudaMemsetAsync(z, 0, 4 * n, s), "clear moments");
  }
  if (rc == THC_OK) {
    to_half_kernel<<<blocks(n1), 256, 0, s>>>(n1, m->W1, m->W1h);
    to_half_kernel<<<blocks(n2), 256, 0, s>>>(n2, m->W2, m->W2h);
    rc = mcheck(m, cudaGetLastError(), "half copies");
  }
  if (rc == THC_OK) rc = mcheck(m, cudaStreamSynchronize(s), "mlp init sync");
  if (rc != THC_OK) {
    for (void* p : m->owned) cudaFree(p);
    delete m;
    return rc;
  }
  *out = m;
  return THC_OK;
}

int thc_mlp_forward(thc_mlp* m, int batch, const float* X, float* Y) {
  if (!m || !X || !Y || batch < 1 || batch > m->max_batch) return mfail(m, THC_EINVAL, "thc_mlp_forward: bad argument");
  THC_TRY(mlp_forward(m, batch, X));
  return mcheck(m, cudaMemcpyAsync(Y, m->Y, 4ull * batch * m->dout, cudaMemcpyDeviceToDevice, m->stream), "copy Y");
}

int thc_mlp_gradients(thc_mlp* m, int batch, const float* X, const float* T, double* loss, float* gW1, float* gb1,
                      float* gW2, float* gb2) {
  if (!m || !X || !T || batch < 1 || batch > m->max_batch) return mfail(m, THC_EINVAL, "thc_mlp_gradients: bad argument");
  THC_TRY(mlp_forward(m, batch, X));
  THC_TRY(mlp_backward(m, batch, X, T));
  const cudaStream_t s = m->stream;
  auto cp = [&](float* dst, const float* src, size_t n) {
    return dst ? mcheck(m, cudaMemcpyAsync(dst, src, 4 * n, cudaMemcpyDefault, s), "copy gradient") : THC_OK;
  };
  THC_TRY(cp(gW1, m->gW1, (size_t)m->H * m->din));
  THC_TRY(cp(gb1, m->gb1, m->H));
  THC_TRY(cp(gW2, m->gW2, (size_t)m->dout * m->H));
  THC_TRY(cp(gb2, m->gb2, m->dout));
  double l = 0.0;
  THC_TRY(mcheck(m, cudaMemcpyAsync(&l, m->loss, 8, cudaMemcpyDeviceToHost, s), "copy loss"));
  THC_TRY(mcheck(m, cudaStreamSynchronize(s), "gradients sync"));
  if (loss) *loss = l / ((double)batch * m->dout);
  return THC_OK;
}

int thc_mlp_train(thc_mlp* m, int n_samples, const float* X, const float* T, int steps, int batch, double lr,
                  double* final_loss) {
  if (!m || !X || !T || n_samples < 1 || steps < 1 || batch < 1)
    return mfail(m, THC_EINVAL, "thc_mlp_train: bad argument");
  batch = std::min(std::min(batch, n_samples), m->max_batch);
  const int nb = (n_samples + batch - 1) / batch;
  for (int st = 0; st < steps; ++st) {
    const int b = st % nb;                 // mini-batches in a fixed cyclic order
    const int off = b * batch, cnt = std::min(batch, n_samples - off);
    const float* xb = X + (long long)off * m->din;
    const float* tb = T + (long long)off * m->dout;
    THC_TRY(mlp_forward(m, cnt, xb));
    THC_TRY(mlp_backward(m, cnt, xb, tb));
    THC_TRY(mlp_adam(m, (float)lr));
  }
  if (final_loss) {
    double l = 0.0;
    THC_TRY(mcheck(m, cudaMemcpyAsync(&l, m->loss, 8, cudaMemcpyDeviceToHost, m->stream), "copy loss"));
    THC_TRY(mcheck(m, cudaStreamSynchronize(m->stream), "train sync"));
    const int last = (steps - 1) % nb;
    const int cnt = std::min(batch, n_samples - last * batch);
    *final_loss = l / ((double)cnt * m->dout);
  }
  return THC_OK;
}

int thc_mlp_get_weights(thc_mlp* m, float* W1, float* b1, float* W2, float* b2) {
  if (!m) return thc::fail(nullptr, THC_EINVAL, "thc_mlp_get_weights: NULL context");
  const cudaStream_t s = m->stream;
  auto cp = [&](float* dst, const float* src, size_t n) {
    return dst ? mcheck(m, cudaMemcpyAsync(dst, src, 4 * n, cudaMemcpyDefault, s), "copy weights") : THC_OK;
  };
  THC_TRY(cp(W1, m->W1, (size_t)m->H * m->din));
  THC_TRY(cp(b1, m->b1, m->H));
  THC_TRY(cp(W2, m->W2, (size_t)m->dout * m->H));
  THC_TRY(cp(b2, m->b2, m->dout));
  return mcheck(m, cudaStreamSynchronize(s), "weights sync");
}

void thc_mlp_destroy(thc_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  for (void* p : m->owned) cudaFree(p);
  delete m;
}

}  // extern "C"

// ================================================================= proposer
struct thc_proposer {
  int n = 0, n_tau = 0, L = 0, max_hist = 0, count = 0;
  long long n2 = 0;
  cudaStream_t stream = nullptr;
  double *U_tau = nullptr, *fit_tau = nullptr;  // n_tau x L, L x n_tau
  double* hist = nullptr;                       // max_hist x L x n2 coefficient ring
  double* prop = nullptr;                       // L x n2 proposal coefficients
  float *X = nullptr, *T = nullptr;             // training samples
  double* red = nullptr;                        // reduction scratch
  thc_mlp* mlp = nullptr;
  double s_c = 1.0, s_d = 1.0;
  std::vector<void*> owned;
  std::string err;
};

namespace {

using thc::f64::View;

int pfail(thc_proposer* p, int code, const std::string& msg) {
  if (p) p->err = msg;
  return thc::fail(nullptr, code, msg);
}
int pcheck(thc_proposer* p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return THC_OK;
  return pfail(p, e == cudaErrorMemoryAllocation ? THC_ENOMEM : THC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct StoreD {
  double* p;
  long long ld;
  double alpha;
  __device__ void operator()(long long, long long m, long long c, double v) const { p[m * ld + c] = alpha * v; }
};

double* slot(thc_proposer* p, int k) { return p->hist + (long long)(k % p->max_hist) * p->L * p->n2; }

// rms of a L x n2 array (or of the difference of two), one CTA, fixed order
__global__ void rms_kernel(long long len, const double* __restrict__ a, const double* __restrict__ b, double* out) {
  double acc = 0.0;
  for (long long i = threadIdx.x; i < len; i += blockDim.x) {
    const double x = b ? a[i] - b[i] : a[i];
    acc = fma(x, x, acc);
  }
  __shared__ double red[32];
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if (threadIdx.x == 0) out[0] = sqrt(acc / (double)max(len, 1LL));
  }
}

// X[s][l] = cj[l][e] / s_c, X[s][L + l] = (cj - cjm)[l][e] / s_d, T[s][l] = (cl - cj)[l][e] / s_d, s = s0 + e
__global__ void samples_kernel(int L, long long n2, const double* __restrict__ cj, const double* __restrict__ cjm,
                               const double* __restrict__ cl, double isc, double isd, float* __restrict__ X,
                               float* __restrict__ T, long long s0) {
  const long long total = (long long)L * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long l = i / n2, e = i - l * n2, s = s0 + e;
    X[s * 2 * L + l] = (float)(cj[i] * isc);
    X[s * 2 * L + L + l] = (float)((cj[i] - cjm[i]) * isd);
    if (T) T[s * L + l] = cl ? (float)((cl[i] - cj[i]) * isd) : 0.f;
  }
}

// prop[l][e] = c[l][e] + s_d Y[e][l]
__global__ void apply_kernel(int L, long long n2, const double* __restrict__ c, const float* __restrict__ Y, double sd,
                             double* __restrict__ prop) {
  const long long total = (long long)L * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long l = i / n2, e = i - l * n2;
    prop[i] = c[i] + sd * (double)Y[e * L + l];
  }
}

int pblocks(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

extern "C" {

int thc_proposer_init(thc_proposer** out, int n_ao, int n_tau, int n_l, const double* U_tau, const double* fit_tau,
                      int hidden, int max_hist, const float* W1, const float* b1, const float* W2, const float* b2,
                      void* stream) {
  if (!out) return thc::fail(nullptr, THC_EINVAL, "thc_proposer_init: NULL out-pointer");
  *out = nullptr;
  if (n_ao < 1 || n_tau < 1 || n_l < 1 || hidden < 1 || max_hist < 3 || !U_tau || !fit_tau)
    return thc::fail(nullptr, THC_EINVAL, "thc_proposer_init: bad sizes (max_hist >= 3) or NULL matrices");
  thc_proposer* p = new (std::nothrow) thc_proposer();
  if (!p) return thc::fail(nullptr, THC_ENOMEM, "thc_proposer_init: host allocation");
  p->n = n_ao, p->n_tau = n_tau, p->L = n_l, p->max_hist = max_hist, p->n2 = (long long)n_ao * n_ao;
  p->stream = (cudaStream_t)stream;
  const size_t L = n_l, n2 = p->n2, ns = (size_t)(max_hist - 2) * n2;
  int rc = THC_OK;
  auto A = [&](void** q, size_t bytes, const char* w) {
    if (rc != THC_OK) return;
    if (cudaMalloc(q, std::max<size_t>(bytes, 8)) != cudaSuccess) {
      cudaGetLastError();
      rc = pfail(p, THC_ENOMEM, std::string("cudaMalloc ") + w);
      return;
    }
    p->owned.push_back(*q);
  };
  A((void**)&p->U_tau, 8 * n_tau * L, "U_tau");
  A((void**)&p->fit_tau, 8 * L * n_tau, "fit_tau");
  A((void**)&p->hist, 8 * (size_t)max_hist * L * n2, "history");
  A((void**)&p->prop, 8 * L * n2, "proposal");
  A((void**)&p->X, 4 * ns * 2 * L, "samples X");
  A((void**)&p->T, 4 * ns * L, "samples T");
  A((void**)&p->red, 8 * (size_t)(max_hist + 4), "scratch");
  if (rc == THC_OK) rc = pcheck(p, cudaMemcpyAsync(p->U_tau, U_tau, 8 * n_tau * L, cudaMemcpyDefault, p->stream), "U_tau");
  if (rc == THC_OK) rc = pcheck(p, cudaMemcpyAsync(p->fit_tau, fit_tau, 8 * L * n_tau, cudaMemcpyDefault, p->stream), "fit");
  if (rc == THC_OK) rc = thc_mlp_init(&p->mlp, 2 * n_l, hidden, n_l, (int)ns, W1, b1, W2, b2, stream);
  if (rc == THC_OK) rc = pcheck(p, cudaStreamSynchronize(p->stream), "proposer init sync");
  if (rc != THC_OK) {
    if (p->mlp) thc_mlp_destroy(p->mlp);
    for (void* q : p->owned) cudaFree(q);
    delete p;
    return rc;
  }
  *out = p;
  return THC_OK;
}

int thc_proposer_observe(thc_proposer* p, const double* Sigma_tau) {
  if (!p || !Sigma_tau) return pfail(p, THC_EINVAL, "thc_proposer_observe: bad argument");
  const long long L = p->L, nt = p->n_tau, n2 = p->n2;
  double* c = slot(p, p->count);
  const dim3 grid((unsigned)((L + 63) / 64), (unsigned)((n2 + 63) / 64), 1);
  thc::f64::gemm_kernel<true, false><<<grid, thc::f64::NT, 0, p->stream>>>(
      L, n2, nt, View{p->fit_tau, 0, nt, 1}, View{Sigma_tau, 0, n2, 1}, StoreD{c, n2, 1.0});
  THC_TRY(pcheck(p, cudaGetLastError(), "coefficients"));
  p->count += 1;
  return THC_OK;
}

int thc_proposer_count(const thc_proposer* p) { return p ? p->count : 0; }

int thc_proposer_reset(thc_proposer* p) {
  if (!p) return thc::fail(nullptr, THC_EINVAL, "thc_proposer_reset: NULL proposer");
  p->count = 0;  // trajectory forgotten, network weights and scales kept
  return THC_OK;
}

int thc_proposer_train(thc_proposer* p, int steps, int batch, double lr, double* final_loss) {
  if (!p || steps < 1) return pfail(p, THC_EINVAL, "thc_proposer_train: bad argument");
  const int k = p->count;  // iterates 0..k-1 observed; latest k-1
  const int first = std::max(1, k - (p->max_hist - 1));
  if (k < 3) return pfail(p, THC_EINVAL, "thc_proposer_train: needs at least three observed iterates");
  const long long L = p->L, n2 = p->n2, len = L * n2;
  double* latest = slot(p, k - 1);
  // s_c from the latest iterate; every pair (j) is scaled by its own change c_j - c_{j-1}, as a
  // proposal made at that point would be
  rms_kernel<<<1, 1024, 0, p->stream>>>(len, latest, nullptr, p->red);
  for (int j = first; j <= k - 2; ++j)
    rms_kernel<<<1, 1024, 0, p->stream>>>(len, slot(p, j), slot(p, j - 1), p->red + 1 + (j - first));
  std::vector<double> h(1 + std::max(0, k - 1 - first));
  THC_TRY(pcheck(p, cudaMemcpyAsync(h.data(), p->red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, p->stream),
                 "scales"));
  THC_TRY(pcheck(p, cudaStreamSynchronize(p->stream), "scales sync"));
  p->s_c = h[0] > 0 ? h[0] : 1.0;
  long long ns = 0;
  for (int j = first; j <= k - 2; ++j) {  // pairs (c_j, c_{j-1}) -> c_latest - c_j
    const double sd = h[1 + (j - first)];
    if (!(sd > 0)) continue;
    samples_kernel<<<pblocks(len), 256, 0, p->stream>>>((int)L, n2, slot(p, j), slot(p, j - 1), latest, 1.0 / p->s_c,
                                                        1.0 / sd, p->X, p->T, ns);
    THC_TRY(pcheck(p, cudaGetLastError(), "samples"));
    ns += n2;
  }
  if (ns == 0) return pfail(p, THC_EINVAL, "thc_proposer_train: the observed iterates do not change");
  return thc_mlp_train(p->mlp, (int)ns, p->X, p->T, steps, batch, lr, final_loss);
}

int thc_proposer_propose(thc_proposer* p, double* Sigma_tau) {
  if (!p || !Sigma_tau) return pfail(p, THC_EINVAL, "thc_proposer_propose: bad argument");
  const int k = p->count;
  if (k < 2) return pfail(p, THC_EINVAL, "thc_proposer_propose: needs at least two observed iterates");
  const long long L = p->L, n2 = p->n2, len = L * n2, nt = p->n_tau;
  double* c = slot(p, k - 1);
  // inputs and outputs are scaled by the current iterate and its last change
  rms_kernel<<<1, 1024, 0, p->stream>>>(len, c, nullptr, p->red);
  rms_kernel<<<1, 1024, 0, p->stream>>>(len, c, slot(p, k - 2), p->red + 1);
  double h[2];
  THC_TRY(pcheck(p, cudaMemcpyAsync(h, p->red, 16, cudaMemcpyDeviceToHost, p->stream), "scales"));
  THC_TRY(pcheck(p, cudaStreamSynchronize(p->stream), "scales sync"));
  p->s_c = h[0] > 0 ? h[0] : 1.0;
  p->s_d = h[1] > 0 ? h[1] : 1.0;
  samples_kernel<<<pblocks(len), 256, 0, p->stream>>>((int)L, n2, c, slot(p, k - 2), nullptr, 1.0 / p->s_c,
                                                      1.0 / p->s_d, p->X, nullptr, 0);
  THC_TRY(pcheck(p, cudaGetLastError(), "features"));
  THC_TRY(mlp_forward(p->mlp, (int)n2, p->X));
  apply_kernel<<<pblocks(len), 256, 0, p->stream>>>((int)L, n2, c, p->mlp->Y, p->s_d, p->prop);
  THC_TRY(pcheck(p, cudaGetLastError(), "apply"));
  const dim3 grid((unsigned)((nt + 63) / 64), (unsigned)((n2 + 63) / 64), 1);
  thc::f64::gemm_kernel<true, false><<<grid, thc::f64::NT, 0, p->stream>>>(
      nt, n2, L, View{p->U_tau, 0, L, 1}, View{p->prop, 0, n2, 1}, StoreD{Sigma_tau, n2, 1.0});
  THC_TRY(pcheck(p, cudaGetLastError(), "proposal to tau"));
  return pcheck(p, cudaStreamSynchronize(p->stream), "propose sync");
}

// ---------------------------------------------------------------- resumable state
// Layout: StateHeader, then the FP32 arrays of the network in the order W1 b1 W2 b2 and
// the Adam moments mW1 vW1 mb1 vb1 mW2 vW2 mb2 vb2, then the observed coefficient window
// (iterates max(0, count - max_hist) .. count - 1, each n_l x n_ao^2 FP64).
namespace {

struct StateHeader {
  char magic[8];
  int32_t n, n_tau, L, H, max_hist, count;
  int64_t t;
  double s_c, s_d;
};

constexpr char kStateMagic[8] = {'T', 'H', 'C', 'P', 'R', 'O', 'P', '1'};

struct StateArray {
  float* p;
  size_t n;
};

std::vector<StateArray> state_arrays(thc_proposer* p) {
  thc_mlp* m = p->mlp;
  const size_t n1 = (size_t)m->H * m->din, n2 = (size_t)m->dout * m->H, H = m->H, D = m->dout;
  return {{m->W1, n1}, {m->b1, H},  {m->W2, n2},  {m->b2, D},  {m->mW1, n1}, {m->vW1, n1},
          {m->mb1, H}, {m->vb1, H}, {m->mW2, n2}, {m->vW2, n2}, {m->mb2, D},  {m->vb2, D}};
}

size_t state_bytes(thc_proposer* p) {
  size_t b = sizeof(StateHeader);
  for (const StateArray& a : state_arrays(p)) b += 4 * a.n;
  const int window = std::min(p->count, p->max_hist);
  return b + 8 * (size_t)window * p->L * p->n2;
}

}  // namespace

int thc_proposer_state_size(const thc_proposer* p, size_t* bytes) {
  if (!p || !bytes) return thc::fail(nullptr, THC_EINVAL, "thc_proposer_state_size: NULL argument");
  *bytes = state_bytes(const_cast<thc_proposer*>(p));
  return THC_OK;
}

int thc_proposer_save_state(thc_proposer* p, void* buf, size_t bytes) {
  if (!p || !buf) return thc::fail(nullptr, THC_EINVAL, "thc_proposer_save_state: NULL argument");
  if (bytes < state_bytes(p)) return pfail(p, THC_EINVAL, "thc_proposer_save_state: buffer too small");
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.n = p->n, h.n_tau = p->n_tau, h.L = p->L, h.H = p->mlp->H, h.max_hist = p->max_hist, h.count = p->count;
  h.t = p->mlp->t, h.s_c = p->s_c, h.s_d = p->s_d;
  uint8_t* out = static_cast<uint8_t*>(buf);
  std::memcpy(out, &h, sizeof h);
  size_t off = sizeof h;
  for (const StateArray& a : state_arrays(p)) {
    THC_TRY(pcheck(p, cudaMemcpyAsync(out + off, a.p, 4 * a.n, cudaMemcpyDeviceToHost, p->stream), "save weights"));
    off += 4 * a.n;
  }
  const size_t slot_bytes = 8 * (size_t)p->L * p->n2;
  for (int k = std::max(0, p->count - p->max_hist); k < p->count; ++k, off += slot_bytes)
    THC_TRY(pcheck(p, cudaMemcpyAsync(out + off, slot(p, k), slot_bytes, cudaMemcpyDeviceToHost, p->stream),
                   "save window"));
  return pcheck(p, cudaStreamSynchronize(p->stream), "save sync");
}

int thc_proposer_load_state(thc_proposer* p, const void* buf, size_t bytes) {
  if (!p || !buf) return thc::fail(nullptr, THC_EINVAL, "thc_proposer_load_state: NULL argument");
  StateHeader h{};
  if (bytes < sizeof h) return pfail(p, THC_EINVAL, "thc_proposer_load_state: buffer too small");
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.n != p->n || h.n_tau != p->n_tau || h.L != p->L ||
      h.H != p->mlp->H || h.max_hist != p->max_hist || h.count < 0)
    return pfail(p, THC_EINVAL, "thc_proposer_load_state: not a state of a proposer of these sizes");
  const int saved_count = p->count;
  p->count = h.count;  // state_bytes sizes the window by count
  const size_t need = state_bytes(p);
  p->count = saved_count;
  if (bytes < need) return pfail(p, THC_EINVAL, "thc_proposer_load_state: buffer too small");
  const uint8_t* in = static_cast<const uint8_t*>(buf);
  size_t off = sizeof h;
  for (const StateArray& a : state_arrays(p)) {
    THC_TRY(pcheck(p, cudaMemcpyAsync(a.p, in + off, 4 * a.n, cudaMemcpyHostToDevice, p->stream), "load weights"));
    off += 4 * a.n;
  }
  const size_t slot_bytes = 8 * (size_t)p->L * p->n2;
  for (int k = std::max(0, h.count - p->max_hist); k < h.count; ++k, off += slot_bytes)
    THC_TRY(pcheck(p, cudaMemcpyAsync(slot(p, k), in + off, slot_bytes, cudaMemcpyHostToDevice, p->stream),
                   "load window"));
  thc_mlp* m = p->mlp;
  const long long n1 = (long long)m->H * m->din, n2 = (long long)m->dout * m->H;
  to_half_kernel<<<blocks(n1), 256, 0, p->stream>>>(n1, m->W1, m->W1h);
  to_half_kernel<<<blocks(n2), 256, 0, p->stream>>>(n2, m->W2, m->W2h);
  THC_TRY(pcheck(p, cudaGetLastError(), "half copies"));
  THC_TRY(pcheck(p, cudaStreamSynchronize(p->stream), "load sync"));
  p->count = h.count;
  m->t = h.t;
  p->s_c = h.s_c;
  p->s_d = h.s_d;
  return THC_OK;
}

const char* thc_proposer_last_error(const thc_proposer* p) { return p ? p->err.c_str() : ""; }

void thc_proposer_destroy(thc_proposer* p) {
  if (!p) return;
  if (p->mlp) thc_mlp_destroy(p->mlp);
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (void* q : p->owned) cudaFree(q);
  delete p;
}

}  // extern "C"
