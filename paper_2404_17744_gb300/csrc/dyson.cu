// Dyson step of the self-consistency loop on the GPU, in FP64 (Sec. II.A,
// Eq. Dyson in a non-orthogonal AO basis):
//
//   Sigma(tau_k) --fit--> sigma_l --> Sigma(i w_m)
//   G(i w_m) = [(i w_m + mu) S - F - Sigma(i w_m)]^{-1}      for every sampled w_m
//   mu such that the electron count per spin Tr[gamma S] = n_elec,
//       gamma = -G(beta^-) = -sum_l u_l(beta) g_l
//   G(i w_m) --fit--> g_l --> G(tau_k)
//
// The tau <-> i w transforms are the sparse-sampling matrices of an IR basis
// (supplied by the caller); they run in the DFMA contraction tile.  The
// inversions are an in-place Gauss-Jordan elimination, a cluster of several
// CTAs per frequency (each owns a block of rows; FP64 is DFMA-bound on GB300,
// so the matrices are spread over as many SMs as the device holds clusters):
// Im[(i w + mu) S - F - Sigma(i w)] = w S - Im Sigma(i w) is
// definite for a causal self-energy, so every leading principal minor is
// non-singular and no pivoting is needed.  When the sampled frequencies come
// in pairs w, -w (the Matsubara sampling of an IR basis does), only the
// positive half is inverted: for real S, F and Sigma(tau), G(-i w) is the
// complex conjugate of G(i w).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "dfma_tile.cuh"
#include "thc_internal.cuh"
#include "thc_dyson.h"

struct thc_dyson {
  int n = 0, n_tau = 0, n_iw = 0, L = 0;
  double beta = 0.0;
  cudaStream_t stream = nullptr;
  std::vector<double> iw;          // host copy of the frequencies
  std::vector<double> cre, cim;    // c_m = sum_l u_l(beta) fit_iw[l, m]
  std::vector<double> parity;      // p_l = u_l(0) / u_l(beta) (+-1)
  std::vector<double> ubeta;
  // device
  double *S = nullptr, *F = nullptr;
  double *U_tau = nullptr, *fit_tau = nullptr;          // n_tau x L, L x n_tau
  double *Uiw_re = nullptr, *Uiw_im = nullptr;          // n_iw x L
  double *fit_re = nullptr, *fit_im = nullptr;          // L x n_iw
  double *fold_re = nullptr, *fold_im = nullptr;        // L x n_iw/2: fit_iw folded onto the positive half
  double *ubeta_d = nullptr, *parity_d = nullptr;       // L
  double *sig_l = nullptr;                              // L x n^2
  double *Siw = nullptr;                                // n_iw x n^2 x 2 (interleaved complex)
  double *Giw = nullptr;                                // n_iw x n^2 x 2
  double *g_l = nullptr;                                // L x n^2 (real part)
  double *tr = nullptr;                                 // n_iw x 2 partial traces
  double *part = nullptr;                               // per-block partial sums of the energy contraction
  bool half = false;                                    // frequencies in pairs (w_m = -w_{n_iw-1-m}): invert m >= n_iw/2
  // Gauss-Jordan launch plan for the gj_count matrices of a set: the first gj_first with
  // clusters of gj_cs[0] CTAs (rows resident in shared memory if gj_res[0]), the rest with
  // gj_cs[1] / gj_res[1]
  long long gj_count = 0, gj_first = 0;
  int gj_cs[2] = {1, 1};
  bool gj_res[2] = {false, false};
  double *scal = nullptr;                               // small scalar scratch
  double *work = nullptr;                               // n_iw x n^2 x 2: G S (count slope), H G (commutator)
  double *work2 = nullptr;                              // n_iw x n^2 x 2: S G (commutator, allocated on first use)
  double *trq = nullptr;                                // n_iw x 2: Tr[(G S)^2]
  int evals = 0;                                        // N(mu) evaluations of the last solve
  std::vector<void*> owned;
  std::string err;
};

namespace {

using thc::f64::BM;
using thc::f64::BN;
using thc::f64::NT;
using thc::f64::View;

int dfail(thc_dyson* d, int code, const std::string& msg) {
  if (d) d->err = msg;
  return thc::fail(nullptr, code, msg);
}

int dcheck(thc_dyson* d, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return THC_OK;
  return dfail(d, e == cudaErrorMemoryAllocation ? THC_ENOMEM : THC_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

int dalloc(thc_dyson* d, double** p, size_t count, const char* what) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, sizeof(double) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return dfail(d, THC_ENOMEM, std::string("cudaMalloc ") + what);
  }
  d->owned.push_back(*p);
  return THC_OK;
}

// C(b) (+)= alpha * A(b) B(b) in the DFMA tile.
struct AccEpi {
  double* p;
  long long sb, sr, sc;
  double alpha;
  bool accumulate;
  __device__ __forceinline__ void operator()(long long b, long long m, long long c, double v) const {
    double* q = p + b * sb + m * sr + c * sc;
    *q = accumulate ? fma(alpha, v, *q) : alpha * v;
  }
};

template <bool AK, bool BK_>
int gemm(thc_dyson* d, long long M, long long Nn, long long K, const View& a, const View& b, const AccEpi& e,
         const char* what, long long batch = 1) {
  const dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Nn + BN - 1) / BN), (unsigned)batch);
  thc::f64::gemm_kernel<AK, BK_><<<grid, NT, 0, d->stream>>>(M, Nn, K, a, b, e);
  return dcheck(d, cudaGetLastError(), what);
}

// A_m = (i w_m + mu) S - F - Sigma(i w_m), interleaved complex.
__global__ void build_kernel(int n, int n_iw, const double* __restrict__ iw, double mu, const double* __restrict__ S,
                             const double* __restrict__ F, const double* __restrict__ Siw, double* __restrict__ A) {
  const long long nn = (long long)n * n, total = nn * n_iw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long m = i / nn, e = i - m * nn;
    const double s = S[e];
    A[2 * i] = mu * s - F[e] - Siw[2 * i];
    A[2 * i + 1] = iw[m] * s - Siw[2 * i + 1];
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// v - f r as four chained FMAs (the FP64 pipe is the bound of the elimination)
__device__ __forceinline__ double2 cfms(double2 f, double2 r, double2 v) {
  return make_double2(fma(f.y, r.y, fma(-f.x, r.x, v.x)), fma(-f.y, r.x, fma(-f.x, r.y, v.y)));
}

// In-place Gauss-Jordan inverse of matrix m0 + blockIdx.x / CS (n x n complex, no
// pivoting), one cluster of CS CTAs per matrix; CTA rank c owns rows
// [c h, min(n, (c + 1) h)), h = ceil(n / CS).  With resident != 0 a CTA keeps its
// rows in shared memory from the first step to the last (when h n complex values
// fit); otherwise they stay in global memory (L2).
//
// Step k uses the scaled pivot row r_j = a_kj / a_kk (r_k = 1 / a_kk), which every
// CTA holds in one of two shared-memory row buffers: each CTA reads and clears
// column k of its rows, then updates them,
//   a_ij -= a_ik r_j (i != k; column k becomes -a_ik / a_kk),  a_kj = r_j,
// and one cluster barrier ends the step.  Look-ahead: during step k the last warp
// of the CTA that owns row k + 1 updates that row first, forms 1 / a_{k+1,k+1}
// (one lane: FP64 division is costly on this GPU), and writes the scaled row into
// the other row buffer of every CTA of the cluster (distributed shared memory),
// while the other warps update the remaining rows.  The buffers alternate, so a
// buffer is written only after every CTA has finished the step that read it.
__global__ void __launch_bounds__(1024) gj_cluster_kernel(int n, int m0, int resident, double2* __restrict__ A0) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int h = (n + CS - 1) / CS, r0 = rank * h, nr = max(0, min(n, r0 + h) - r0);
  extern __shared__ double2 sh[];
  double2* rowbuf = sh;          // [2][n] scaled pivot rows, written by their owner
  double2* colk = sh + 2 * n;    // [h] column k of this CTA's rows
  double2* A = A0 + (long long)(m0 + blockIdx.x / CS) * n * n;
  double2* blk = A + (long long)r0 * n;  // this CTA's rows, row stride n
  const long long cnt = (long long)nr * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int la_warp = nwarp - 1;
  if (resident) {
    double2* s_rows = colk + h;
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) s_rows[e] = blk[e];
    blk = s_rows;
  }
  // one warp: scale row kk (held in src) by 1 / src[kk] into row buffer kk & 1 of every CTA
  auto publish = [&](int kk, const double2* src) {
    double px = 0.0, py = 0.0;
    if (lane == 0) {
      const double2 p = src[kk];
      const double inv = 1.0 / (p.x * p.x + p.y * p.y);
      px = p.x * inv;
      py = -p.y * inv;
    }
    const double2 ip = make_double2(__shfl_sync(0xffffffffu, px, 0), __shfl_sync(0xffffffffu, py, 0));
    for (int j = lane; j < n; j += 32) {
      const double2 v = (j == kk) ? ip : cmul(src[j], ip);
      for (int c = 0; c < CS; ++c) cluster.map_shared_rank(rowbuf + (kk & 1) * n, c)[j] = v;
    }
  };
  cluster.sync();  // every CTA of the cluster runs (and holds its rows) before remote writes
  if (rank == 0 && warp == la_warp) publish(0, blk);
  cluster.sync();
  for (int k = 0; k < n; ++k) {
    const double2* rowk = rowbuf + (k & 1) * n;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      colk[i] = blk[(long long)i * n + k];
      if (r0 + i != k) blk[(long long)i * n + k] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int kn = k + 1, lin = kn - r0;
    const bool la = kn < n && kn / h == rank;  // this CTA owns the next pivot row
    if (la && warp == la_warp) {
      double2* Ar = blk + (long long)lin * n;
      const double2 f = colk[lin];
      for (int j = lane; j < n; j += 32) Ar[j] = cfms(f, rowk[j], Ar[j]);
      __syncwarp();
      publish(kn, Ar);
    }
    for (int j = lane; j < n; j += 32) {
      const double2 r = rowk[j];
      for (int li = warp; li < nr; li += nwarp) {
        if (la && li == lin) continue;
        double2* a = blk + (long long)li * n + j;
        if (r0 + li == k) {
          *a = r;
        } else {
          *a = cfms(colk[li], r, *a);
        }
      }
    }
    cluster.sync();  // step k done everywhere; row k + 1 published
  }
  if (resident) {
    double2* out = A + (long long)r0 * n;
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) out[e] = blk[e];
  }
}

// G[m] = conj(G[n_iw - 1 - m]) for m < n_iw / 2.
__global__ void mirror_conj_kernel(long long nn, int nw, double2* __restrict__ G) {
  const long long total = nn * (nw / 2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long m = i / nn, e = i - m * nn;
    const double2 v = G[(long long)(nw - 1 - m) * nn + e];
    G[m * nn + e] = make_double2(v.x, -v.y);
  }
}

// t_m = Tr[G_m S] = sum_ij G_m[i][j] S[j][i] (complex), one CTA per m.
__global__ void trace_gs_kernel(int n, const double2* __restrict__ G, const double* __restrict__ S,
                                double* __restrict__ t) {
  const long long m = blockIdx.x, nn = (long long)n * n;
  const double2* g = G + m * nn;
  double re = 0.0, im = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, j = e - i * n;
    const double s = S[j * n + i];
    re = fma(g[e].x, s, re);
    im = fma(g[e].y, s, im);
  }
  __shared__ double r1[32], r2[32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = re;
    r2[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    re = threadIdx.x < (blockDim.x >> 5) ? r1[threadIdx.x] : 0.0;
    im = threadIdx.x < (blockDim.x >> 5) ? r2[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (threadIdx.x == 0) {
      t[2 * m] = re;
      t[2 * m + 1] = im;
    }
  }
}

// q_m = Tr[Y_m Y_m] = sum_ik Y_m[i][k] Y_m[k][i] (complex), one CTA per m.
__global__ void trace_sq_kernel(int n, const double2* __restrict__ Y, double* __restrict__ q) {
  const long long m = blockIdx.x, nn = (long long)n * n;
  const double2* y = Y + m * nn;
  double re = 0.0, im = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const long long i = e / n, k = e - i * n;
    const double2 a = y[e], b = y[k * n + i];
    re = fma(a.x, b.x, fma(-a.y, b.y, re));
    im = fma(a.x, b.y, fma(a.y, b.x, im));
  }
  __shared__ double r1[32], r2[32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = re;
    r2[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    re = threadIdx.x < (blockDim.x >> 5) ? r1[threadIdx.x] : 0.0;
    im = threadIdx.x < (blockDim.x >> 5) ? r2[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (threadIdx.x == 0) {
      q[2 * m] = re;
      q[2 * m + 1] = im;
    }
  }
}

// H_m = F + Sigma(i w_m): F added to the real parts of the interleaved complex matrices.
__global__ void add_real_kernel(long long nn, int nw, const double* __restrict__ F, double* __restrict__ H) {
  const long long total = nn * nw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    H[2 * i] += F[i % nn];
}

// part[2 b], part[2 b + 1]: block b's share of
//   sum_l p_l sum_ij a_l[i][j] b_l[j][i]   and   sum_l ub_l sum_ij a_l[i][j] M[j][i]
// over the rows (l, i) it owns (one warp per row, lanes along j).
__global__ void coef_contract_kernel(int n, int L, const double* __restrict__ a, const double* __restrict__ b,
                                     const double* __restrict__ p, const double* __restrict__ ub,
                                     const double* __restrict__ M, double* __restrict__ part) {
  const long long nn = (long long)n * n, rows = (long long)L * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  double s1 = 0.0, s2 = 0.0;
  for (long long row = (long long)blockIdx.x * nwarp + warp; row < rows; row += (long long)gridDim.x * nwarp) {
    const long long l = row / n, i = row - l * n;
    const double* ar = a + row * n;
    const double* bl = b + l * nn;
    double t1 = 0.0, t2 = 0.0;
    for (int j = lane; j < n; j += 32) {
      const double av = ar[j];
      t1 = fma(av, bl[(long long)j * n + i], t1);
      if (M) t2 = fma(av, M[(long long)j * n + i], t2);
    }
    s1 = fma(p[l], t1, s1);
    s2 = fma(ub[l], t2, s2);
  }
  __shared__ double r1[32], r2[32];
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    r1[warp] = s1;
    r2[warp] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    s1 = threadIdx.x < nwarp ? r1[threadIdx.x] : 0.0;
    s2 = threadIdx.x < nwarp ? r2[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = s1;
      part[2 * blockIdx.x + 1] = s2;
    }
  }
}

// out[0..1] = column sums of part[cnt][2], in a fixed order (one warp).
__global__ void pair_sum_kernel(int cnt, const double* __restrict__ part, double* __restrict__ out) {
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < cnt; i += 32) {
    s1 += part[2 * i];
    s2 += part[2 * i + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (threadIdx.x == 0) {
    out[0] = s1;
    out[1] = s2;
  }
}
constexpr int kEnergyBlocks = 296;  // 2 per SM

int blocks_for(long long total) { return (int)std::min<long long>((total + 255) / 256, 152LL * 32); }

// sigma_l = fit_tau Sigma(tau);  Sigma(i w_m) = U_iw sigma_l (interleaved complex) for m >= m_first
int sigma_to_iw(thc_dyson* d, const double* Sig_tau, long long m_first = 0) {
  const long long n2 = (long long)d->n * d->n, L = d->L, nt = d->n_tau, nw = d->n_iw - m_first;
  THC_TRY(gemm<true, false>(d, L, n2, nt, View{d->fit_tau, 0, nt, 1}, View{Sig_tau, 0, n2, 1},
                            AccEpi{d->sig_l, 0, n2, 1, 1.0, false}, "sigma_l"));
  double* out = d->Siw + 2 * m_first * n2;
  THC_TRY(gemm<true, false>(d, nw, n2, L, View{d->Uiw_re + m_first * L, 0, L, 1}, View{d->sig_l, 0, n2, 1},
                            AccEpi{out, 0, 2 * n2, 2, 1.0, false}, "Sigma(iw) re"));
  return gemm<true, false>(d, nw, n2, L, View{d->Uiw_im + m_first * L, 0, L, 1}, View{d->sig_l, 0, n2, 1},
                           AccEpi{out + 1, 0, 2 * n2, 2, 1.0, false}, "Sigma(iw) im");
}

// First frequency the inversions use: the positive half when the frequencies come in pairs.
long long first_inverted(const thc_dyson* d) { return d->half ? d->n_iw / 2 : 0; }

// Dynamic shared memory of gj_cluster_kernel: two pivot-row buffers and a column, plus the
// CTA's rows when they are resident.
size_t gj_smem(int n, int cs, bool resident) {
  const size_t h = (size_t)((n + cs - 1) / cs);
  return sizeof(double2) * (2 * (size_t)n + h + (resident ? h * (size_t)n : 0));
}
constexpr size_t kGjSmemMax = 232448;  // 227 KB per CTA

// Launch plan of the Gauss-Jordan kernel.  A set's time is the sum over its launches of
// the rows per CTA times the waves of resident clusters (rows kept in global memory, L2,
// counted twice).  Candidates: one cluster size for every matrix, or whole waves of one
// size followed by the remaining matrices with another (a last partial wave of small
// clusters leaves most SMs idle; larger clusters spread those matrices over them).
int choose_gj_cluster(thc_dyson* d) {
  THC_TRY(thc::per_device(reinterpret_cast<const void*>(gj_cluster_kernel), nullptr, [&](int, int*) {
    return dcheck(d, cudaFuncSetAttribute(gj_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kGjSmemMax),
                  "Gauss-Jordan shared memory");
  }));
  const long long count = d->half ? d->n_iw / 2 : d->n_iw;
  struct Opt {
    int cs;
    bool res;
    long long q, rows;  // resident clusters, cost of one wave
  };
  std::vector<Opt> opts;
  for (int cs = 1; cs <= 8 && cs <= d->n; ++cs) {
    for (int res = 0; res < 2; ++res) {
      const size_t smem = gj_smem(d->n, cs, res != 0);
      if (smem > kGjSmemMax) continue;
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)cs;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(cs * std::max<long long>(1, count)), 1, 1);
      cfg.blockDim = dim3(1024, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int q = 0;
      if (cudaOccupancyMaxActiveClusters(&q, gj_cluster_kernel, &cfg) != cudaSuccess || q < 1) {
        cudaGetLastError();
        continue;
      }
      opts.push_back(Opt{cs, res != 0, q, (long long)((d->n + cs - 1) / cs) * (res ? 1 : 2)});
    }
  }
  if (opts.empty()) return dfail(d, THC_EINVAL, "no cluster shape of the Gauss-Jordan kernel fits this device");
  auto waves = [](long long m, long long q) { return (m + q - 1) / q; };
  long long best = -1;
  for (const Opt& a : opts) {
    const long long single = waves(count, a.q) * a.rows;
    if (best < 0 || single < best) {  // ties: the earlier (smaller) cluster
      best = single;
      d->gj_first = count;
      d->gj_cs[0] = d->gj_cs[1] = a.cs;
      d->gj_res[0] = d->gj_res[1] = a.res;
    }
    const long long first = (count / a.q) * a.q, rest = count - first;
    if (first == 0 || rest == 0) continue;
    for (const Opt& b : opts) {
      const long long cost = (first / a.q) * a.rows + waves(rest, b.q) * b.rows;
      if (cost < best) {
        best = cost;
        d->gj_first = first;
        d->gj_cs[0] = a.cs;
        d->gj_res[0] = a.res;
        d->gj_cs[1] = b.cs;
        d->gj_res[1] = b.res;
      }
    }
  }
  d->gj_count = count;
  return THC_OK;
}

// Gauss-Jordan inversion of count matrices of d->Giw from m0 on, clusters of cs CTAs each.
int invert_launch(thc_dyson* d, long long m0, long long count, int cs, bool res) {
  if (count <= 0) return THC_OK;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(count * cs), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = gj_smem(d->n, cs, res);
  cfg.stream = d->stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, gj_cluster_kernel, d->n, (int)m0, res ? 1 : 0,
                                           reinterpret_cast<double2*>(d->Giw));
  return dcheck(d, e == cudaSuccess ? cudaGetLastError() : e, "Gauss-Jordan");
}

// The matrices m0 .. m0 + count - 1 by the launch plan (one launch when count is not the
// planned set).
int invert(thc_dyson* d, long long m0, long long count) {
  if (count != d->gj_count) return invert_launch(d, m0, count, d->gj_cs[0], d->gj_res[0]);
  const long long first = std::min(count, d->gj_first);
  THC_TRY(invert_launch(d, m0, first, d->gj_cs[0], d->gj_res[0]));
  return invert_launch(d, m0 + first, count - first, d->gj_cs[1], d->gj_res[1]);
}

// Re sum_m c_m t_m over every frequency from the traces t (interleaved complex) of the
// inverted ones: Tr[gamma S] = -Re sum_m c_m t_m, dN/dmu = Re sum_m c_m q_m; for the
// mirrored half t_{n_iw - 1 - m} = conj(t_m) (likewise q).
double freq_sum(const thc_dyson* d, const double* t) {
  const long long nw = d->n_iw;
  double acc = 0.0;
  for (long long m = first_inverted(d); m < nw; ++m) {
    acc += d->cre[m] * t[2 * m] - d->cim[m] * t[2 * m + 1];
    if (d->half) {
      const long long mm = nw - 1 - m;
      acc += d->cre[mm] * t[2 * m] + d->cim[mm] * t[2 * m + 1];
    }
  }
  return acc;
}

// G(i w_m) at chemical potential mu for every m (the positive half only when the
// frequencies come in pairs); returns the electron count per spin.
int dyson_at(thc_dyson* d, double mu, double* n_out) {
  const long long n = d->n, nn = n * n, nw = d->n_iw;
  const long long m0 = first_inverted(d), cnt = nw - m0;
  const double* iw_d = d->scal + 8 + m0;  // frequencies live after 8 scalar slots
  build_kernel<<<blocks_for(nn * cnt), 256, 0, d->stream>>>((int)n, (int)cnt, iw_d, mu, d->S, d->F,
                                                            d->Siw + 2 * m0 * nn, d->Giw + 2 * m0 * nn);
  THC_TRY(dcheck(d, cudaGetLastError(), "Dyson matrices"));
  THC_TRY(invert(d, m0, cnt));
  trace_gs_kernel<<<(unsigned)cnt, 256, 0, d->stream>>>((int)n, reinterpret_cast<const double2*>(d->Giw) + m0 * nn,
                                                        d->S, d->tr + 2 * m0);
  THC_TRY(dcheck(d, cudaGetLastError(), "Tr[G S]"));
  std::vector<double> t(2 * nw);
  THC_TRY(dcheck(d, cudaMemcpyAsync(t.data() + 2 * m0, d->tr + 2 * m0, sizeof(double) * 2 * cnt,
                                    cudaMemcpyDeviceToHost, d->stream),
                 "copy traces"));
  THC_TRY(dcheck(d, cudaStreamSynchronize(d->stream), "Dyson sync"));
  *n_out = -freq_sum(d, t.data());
  d->evals += 1;
  return THC_OK;
}

// dN/dmu at the G(i w) of the last dyson_at: dG/dmu = -G S G, so dt_m/dmu = -Tr[(G_m S)^2] = -q_m,
// from Y_m = G_m S (real and imaginary parts).
int dyson_slope(thc_dyson* d, double* dn_out) {
  const long long n = d->n, nn = n * n, nw = d->n_iw;
  const long long m0 = first_inverted(d), cnt = nw - m0;
  for (int part = 0; part < 2; ++part)
    THC_TRY(gemm<true, false>(d, n, n, n, View{d->Giw + 2 * m0 * nn + part, 2 * nn, 2 * n, 2}, View{d->S, 0, n, 1},
                              AccEpi{d->work + 2 * m0 * nn + part, 2 * nn, 2 * n, 2, 1.0, false}, "G S", cnt));
  trace_sq_kernel<<<(unsigned)cnt, 256, 0, d->stream>>>((int)n, reinterpret_cast<const double2*>(d->work) + m0 * nn,
                                                        d->trq + 2 * m0);
  THC_TRY(dcheck(d, cudaGetLastError(), "Tr[(G S)^2]"));
  std::vector<double> q(2 * nw);
  THC_TRY(dcheck(d, cudaMemcpyAsync(q.data() + 2 * m0, d->trq + 2 * m0, sizeof(double) * 2 * cnt,
                                    cudaMemcpyDeviceToHost, d->stream),
                 "copy slope traces"));
  THC_TRY(dcheck(d, cudaStreamSynchronize(d->stream), "Dyson slope sync"));
  *dn_out = freq_sum(d, q.data());
  return THC_OK;
}

}  // namespace

extern "C" {

int thc_dyson_init(thc_dyson** out, int n_ao, int n_tau, int n_iw, int n_l, double beta, const double* S,
                   const double* F, const double* U_tau, const double* fit_tau, const double* U_iw,
                   const double* fit_iw, const double* iw, const double* u_beta, const double* u_zero, void* stream) {
  if (!out) return thc::fail(nullptr, THC_EINVAL, "thc_dyson_init: NULL out-pointer");
  *out = nullptr;
  if (n_ao < 1 || n_tau < 1 || n_iw < 1 || n_l < 1 || !(beta > 0))
    return thc::fail(nullptr, THC_EINVAL, "thc_dyson_init: sizes must be >= 1 and beta > 0");
  if (n_ao > 1500) return thc::fail(nullptr, THC_EINVAL, "thc_dyson_init: n_ao above 1500 is not supported");
  if (!S || !F || !U_tau || !fit_tau || !U_iw || !fit_iw || !iw || !u_beta || !u_zero)
    return thc::fail(nullptr, THC_EINVAL, "thc_dyson_init: NULL argument");
  thc_dyson* d = new (std::nothrow) thc_dyson();
  if (!d) return thc::fail(nullptr, THC_ENOMEM, "thc_dyson_init: host allocation");
  d->n = n_ao;
  d->n_tau = n_tau;
  d->n_iw = n_iw;
  d->L = n_l;
  d->beta = beta;
  d->stream = (cudaStream_t)stream;
  auto bail = [&](int rc) {
    for (void* p : d->owned) cudaFree(p);
    delete d;
    return rc;
  };
  const size_t n2 = (size_t)n_ao * n_ao, L = n_l;
  // host-side constants of the transforms
  d->iw.assign(iw, iw + n_iw);
  d->ubeta.assign(u_beta, u_beta + L);
  d->parity.resize(L);
  for (size_t l = 0; l < L; ++l) d->parity[l] = (u_zero[l] * u_beta[l] >= 0.0) ? 1.0 : -1.0;
  d->cre.assign(n_iw, 0.0);
  d->cim.assign(n_iw, 0.0);
  for (int m = 0; m < n_iw; ++m)
    for (size_t l = 0; l < L; ++l) {
      d->cre[m] += u_beta[l] * fit_iw[2 * (l * n_iw + m)];
      d->cim[m] += u_beta[l] * fit_iw[2 * (l * n_iw + m) + 1];
    }
  std::vector<double> a(n_iw * L), b(n_iw * L), c(L * n_iw), e(L * n_iw);
  for (size_t i = 0; i < (size_t)n_iw * L; ++i) {
    a[i] = U_iw[2 * i];
    b[i] = U_iw[2 * i + 1];
    c[i] = fit_iw[2 * i];
    e[i] = fit_iw[2 * i + 1];
  }
  int rc = THC_OK;
  auto up = [&](double** dst, const double* src, size_t cnt, const char* what) {
    if (rc != THC_OK) return;
    rc = dalloc(d, dst, cnt, what);
    if (rc == THC_OK) rc = dcheck(d, cudaMemcpyAsync(*dst, src, sizeof(double) * cnt, cudaMemcpyDefault, d->stream), what);
  };
  up(&d->S, S, n2, "S");
  up(&d->F, F, n2, "F");
  up(&d->U_tau, U_tau, (size_t)n_tau * L, "U_tau");
  up(&d->fit_tau, fit_tau, L * n_tau, "fit_tau");
  up(&d->Uiw_re, a.data(), a.size(), "U_iw re");
  up(&d->Uiw_im, b.data(), b.size(), "U_iw im");
  up(&d->fit_re, c.data(), c.size(), "fit_iw re");
  up(&d->fit_im, e.data(), e.size(), "fit_iw im");
  up(&d->ubeta_d, d->ubeta.data(), L, "u(beta)");
  up(&d->parity_d, d->parity.data(), L, "parity");
  if (rc == THC_OK) rc = dalloc(d, &d->sig_l, L * n2, "sigma_l");
  if (rc == THC_OK) rc = dalloc(d, &d->g_l, L * n2, "g_l");
  if (rc == THC_OK) rc = dalloc(d, &d->Siw, 2 * n2 * n_iw, "Sigma(iw)");
  if (rc == THC_OK) rc = dalloc(d, &d->Giw, 2 * n2 * n_iw, "G(iw)");
  if (rc == THC_OK) rc = dalloc(d, &d->tr, 2 * (size_t)n_iw, "traces");
  if (rc == THC_OK) rc = dalloc(d, &d->trq, 2 * (size_t)n_iw, "slope traces");
  if (rc == THC_OK) rc = dalloc(d, &d->work, 2 * n2 * n_iw, "G S");
  if (rc == THC_OK) rc = dalloc(d, &d->scal, 8 + (size_t)n_iw, "scalars");
  if (rc == THC_OK) rc = dalloc(d, &d->part, 2 * (size_t)kEnergyBlocks, "energy partial sums");
  if (rc == THC_OK)
    rc = dcheck(d, cudaMemcpyAsync(d->scal + 8, iw, sizeof(double) * n_iw, cudaMemcpyDefault, d->stream), "iw");
  if (rc == THC_OK) rc = dcheck(d, cudaStreamSynchronize(d->stream), "dyson init sync");
  // frequencies in pairs (w_m = -w_{n_iw-1-m}, positive in the upper half): invert that half only
  d->half = n_iw % 2 == 0;
  for (int m = n_iw / 2; m < n_iw && d->half; ++m)
    if (!(iw[m] > 0.0) || !(std::fabs(iw[m] + iw[n_iw - 1 - m]) <= 1e-12 * iw[m])) d->half = false;
  if (rc == THC_OK && d->half) {
    // fit_iw folded onto the positive half: Re[f_m G_m + f_mm conj(G_m)] = (Re f_m + Re f_mm) Re G_m
    // - (Im f_m - Im f_mm) Im G_m, mm = n_iw - 1 - m
    const int h = n_iw / 2;
    std::vector<double> fr(L * h), fi(L * h);
    for (size_t l = 0; l < L; ++l)
      for (int j = 0; j < h; ++j) {
        const size_t m = (size_t)(h + j), mm = (size_t)(n_iw - 1) - m;
        fr[l * h + j] = fit_iw[2 * (l * n_iw + m)] + fit_iw[2 * (l * n_iw + mm)];
        fi[l * h + j] = fit_iw[2 * (l * n_iw + m) + 1] - fit_iw[2 * (l * n_iw + mm) + 1];
      }
    up(&d->fold_re, fr.data(), fr.size(), "folded fit_iw re");
    up(&d->fold_im, fi.data(), fi.size(), "folded fit_iw im");
    if (rc == THC_OK) rc = dcheck(d, cudaStreamSynchronize(d->stream), "folded fit_iw sync");
  }
  if (rc == THC_OK) rc = choose_gj_cluster(d);
  if (rc != THC_OK) return bail(rc);
  *out = d;
  return THC_OK;
}

int thc_dyson_solve(thc_dyson* d, const double* Sigma_tau, double n_elec, double* mu, double tol, double* G_tau) {
  if (!d) return thc::fail(nullptr, THC_EINVAL, "thc_dyson_solve: NULL context");
  if (!mu || !G_tau) return dfail(d, THC_EINVAL, "thc_dyson_solve: NULL argument");
  const long long n2 = (long long)d->n * d->n, L = d->L, nt = d->n_tau, nw = d->n_iw;
  d->evals = 0;
  if (Sigma_tau) {
    THC_TRY(sigma_to_iw(d, Sigma_tau, first_inverted(d)));
  } else {
    THC_TRY(dcheck(d, cudaMemsetAsync(d->Siw, 0, sizeof(double) * 2 * n2 * nw, d->stream), "zero Sigma"));
  }
  if (!(tol > 0)) tol = 1e-10;
  // N(mu) is increasing.  Newton steps on the analytic slope dN/dmu (from
  // dG/dmu = -G S G, evaluated with every count that another step follows), each
  // capped at 0.5 Ha, kept inside a bracket once one is known and replaced by
  // bisection when they leave it, when the slope vanishes (mu in a gap) or every
  // fourth step.
  double m = *mu, nm = 0.0, dm = 0.0;
  THC_TRY(dyson_at(d, m, &nm));
  if (std::fabs(nm - n_elec) > tol) THC_TRY(dyson_slope(d, &dm));
  double lo = -INFINITY, hi = INFINITY;
  auto note = [&](double x, double nx) {
    if (nx < n_elec) {
      if (x > lo) lo = x;
    } else if (x < hi) {
      hi = x;
    }
  };
  note(m, nm);
  for (int it = 0; it < 200 && std::fabs(nm - n_elec) > tol; ++it) {
    const bool bracket = std::isfinite(lo) && std::isfinite(hi);
    if (bracket && hi - lo < 1e-15) break;
    double x;
    if (dm > 1e-12 && std::isfinite(dm) && !(bracket && it % 4 == 3)) {
      const double st = (n_elec - nm) / dm;
      x = m + std::min(std::max(st, -0.5), 0.5);
    } else if (bracket) {
      x = 0.5 * (lo + hi);
    } else {
      x = m + (nm < n_elec ? 0.5 : -0.5);  // flat count (a gap) and no bracket yet: walk out
    }
    if (bracket && !(x > lo && x < hi)) x = 0.5 * (lo + hi);
    m = x;
    THC_TRY(dyson_at(d, m, &nm));
    note(m, nm);
    if (std::fabs(nm - n_elec) > tol) THC_TRY(dyson_slope(d, &dm));
  }
  if (std::fabs(nm - n_elec) > 1e3 * tol)
    return dfail(d, THC_EINVAL, "thc_dyson_solve: chemical potential search did not converge");
  *mu = m;
  if (d->half) {
    mirror_conj_kernel<<<blocks_for(n2 * (nw / 2)), 256, 0, d->stream>>>(n2, (int)nw,
                                                                        reinterpret_cast<double2*>(d->Giw));
    THC_TRY(dcheck(d, cudaGetLastError(), "G(-i w)"));
  }
  // g_l = Re[fit_iw G(iw)] ;  G(tau) = U_tau g.  With the frequencies in pairs the sum runs
  // over the positive half with the folded coefficients (fit_m + fit_{n_iw-1-m} on Re G_m,
  // their imaginary parts' difference on Im G_m).
  const long long m0 = first_inverted(d), kw = nw - m0;
  const double* fre = d->half ? d->fold_re : d->fit_re;
  const double* fim = d->half ? d->fold_im : d->fit_im;
  THC_TRY(gemm<true, false>(d, L, n2, kw, View{fre, 0, kw, 1}, View{d->Giw + 2 * m0 * n2, 0, 2 * n2, 2},
                            AccEpi{d->g_l, 0, n2, 1, 1.0, false}, "g_l re"));
  THC_TRY(gemm<true, false>(d, L, n2, kw, View{fim, 0, kw, 1}, View{d->Giw + 2 * m0 * n2 + 1, 0, 2 * n2, 2},
                            AccEpi{d->g_l, 0, n2, 1, -1.0, true}, "g_l im"));
  THC_TRY(gemm<true, false>(d, nt, n2, L, View{d->U_tau, 0, L, 1}, View{d->g_l, 0, n2, 1},
                            AccEpi{G_tau, 0, n2, 1, 1.0, false}, "G(tau)"));
  return dcheck(d, cudaStreamSynchronize(d->stream), "dyson solve sync");
}

int thc_dyson_count(thc_dyson* d, const double* Sigma_tau, double mu, double* n_per_spin, double* dn_dmu) {
  if (!d) return thc::fail(nullptr, THC_EINVAL, "thc_dyson_count: NULL context");
  if (!n_per_spin) return dfail(d, THC_EINVAL, "thc_dyson_count: NULL argument");
  const long long n2 = (long long)d->n * d->n;
  if (Sigma_tau) {
    THC_TRY(sigma_to_iw(d, Sigma_tau, first_inverted(d)));
  } else {
    THC_TRY(dcheck(d, cudaMemsetAsync(d->Siw, 0, sizeof(double) * 2 * n2 * d->n_iw, d->stream), "zero Sigma"));
  }
  THC_TRY(dyson_at(d, mu, n_per_spin));
  return dn_dmu ? dyson_slope(d, dn_dmu) : THC_OK;
}

int thc_dyson_commutator(thc_dyson* d, const double* Sigma_out_tau, double* E_iw) {
  if (!d) return thc::fail(nullptr, THC_EINVAL, "thc_dyson_commutator: NULL context");
  if (!Sigma_out_tau || !E_iw) return dfail(d, THC_EINVAL, "thc_dyson_commutator: NULL argument");
  const long long n = d->n, nn = n * n, nw = d->n_iw;
  if (!d->work2) THC_TRY(dalloc(d, &d->work2, 2 * nn * nw, "S G"));
  // H_m = F + Sigma_out(i w_m) in d->Siw; G_m of the last solve in d->Giw (all frequencies)
  THC_TRY(sigma_to_iw(d, Sigma_out_tau));
  add_real_kernel<<<blocks_for(nn * nw), 256, 0, d->stream>>>(nn, (int)nw, d->F, d->Siw);
  THC_TRY(dcheck(d, cudaGetLastError(), "F + Sigma(iw)"));
  // complex interleaved views: part 0 real, 1 imaginary; batch m
  auto cv = [&](const double* base, int part) { return View{base + part, 2 * nn, 2 * n, 2}; };
  auto ce = [&](double* base, int part, double alpha, bool acc) {
    return AccEpi{base + part, 2 * nn, 2 * n, 2, alpha, acc};
  };
  const View Sv{d->S, 0, n, 1};
  double *H = d->Siw, *G = d->Giw, *P = d->work, *Q = d->work2;
  // P = H G
  THC_TRY(gemm<true, false>(d, n, n, n, cv(H, 0), cv(G, 0), ce(P, 0, 1.0, false), "H G", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, cv(H, 1), cv(G, 1), ce(P, 0, -1.0, true), "H G", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, cv(H, 0), cv(G, 1), ce(P, 1, 1.0, false), "H G", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, cv(H, 1), cv(G, 0), ce(P, 1, 1.0, true), "H G", nw));
  // E = P S
  THC_TRY(gemm<true, false>(d, n, n, n, cv(P, 0), Sv, ce(E_iw, 0, 1.0, false), "H G S", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, cv(P, 1), Sv, ce(E_iw, 1, 1.0, false), "H G S", nw));
  // Q = S G
  THC_TRY(gemm<true, false>(d, n, n, n, Sv, cv(G, 0), ce(Q, 0, 1.0, false), "S G", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, Sv, cv(G, 1), ce(Q, 1, 1.0, false), "S G", nw));
  // E -= Q H
  THC_TRY(gemm<true, false>(d, n, n, n, cv(Q, 0), cv(H, 0), ce(E_iw, 0, -1.0, true), "S G H", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, cv(Q, 1), cv(H, 1), ce(E_iw, 0, 1.0, true), "S G H", nw));
  THC_TRY(gemm<true, false>(d, n, n, n, cv(Q, 0), cv(H, 1), ce(E_iw, 1, -1.0, true), "S G H", nw));
  return gemm<true, false>(d, n, n, n, cv(Q, 1), cv(H, 0), ce(E_iw, 1, -1.0, true), "S G H", nw);
}

int thc_dyson_energy(thc_dyson* d, const double* G_tau, const double* Sigma_tau, double* E_dyn, double* gamma_F,
                     double* n_per_spin) {
  if (!d) return thc::fail(nullptr, THC_EINVAL, "thc_dyson_energy: NULL context");
  if (!G_tau || !Sigma_tau || !E_dyn) return dfail(d, THC_EINVAL, "thc_dyson_energy: NULL argument");
  const long long n2 = (long long)d->n * d->n, L = d->L, nt = d->n_tau;
  // coefficients of G and Sigma
  THC_TRY(gemm<true, false>(d, L, n2, nt, View{d->fit_tau, 0, nt, 1}, View{G_tau, 0, n2, 1},
                            AccEpi{d->g_l, 0, n2, 1, 1.0, false}, "g_l"));
  THC_TRY(gemm<true, false>(d, L, n2, nt, View{d->fit_tau, 0, nt, 1}, View{Sigma_tau, 0, n2, 1},
                            AccEpi{d->sig_l, 0, n2, 1, 1.0, false}, "sigma_l"));
  // E_dyn = -int Tr[G(beta - tau) Sigma(tau)] = -sum_l p_l Tr[g_l sigma_l];  Tr[G(beta^-) F], Tr[G(beta^-) S]
  double h[4];
  coef_contract_kernel<<<kEnergyBlocks, 512, 0, d->stream>>>((int)d->n, (int)L, d->g_l, d->sig_l, d->parity_d,
                                                            d->ubeta_d, d->F, d->part);
  pair_sum_kernel<<<1, 32, 0, d->stream>>>(kEnergyBlocks, d->part, d->scal);
  THC_TRY(dcheck(d, cudaGetLastError(), "energy contraction"));
  coef_contract_kernel<<<kEnergyBlocks, 512, 0, d->stream>>>((int)d->n, (int)L, d->g_l, d->sig_l, d->parity_d,
                                                            d->ubeta_d, d->S, d->part);
  pair_sum_kernel<<<1, 32, 0, d->stream>>>(kEnergyBlocks, d->part, d->scal + 2);
  THC_TRY(dcheck(d, cudaGetLastError(), "count contraction"));
  THC_TRY(dcheck(d, cudaMemcpyAsync(h, d->scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, d->stream), "copy"));
  THC_TRY(dcheck(d, cudaStreamSynchronize(d->stream), "energy sync"));
  *E_dyn = -h[0];
  if (gamma_F) *gamma_F = -h[1];     // Tr[gamma F], gamma = -G(beta^-)
  if (n_per_spin) *n_per_spin = -h[3];
  return THC_OK;
}

int thc_dyson_evals(const thc_dyson* d) { return d ? d->evals : 0; }

// ---------------------------------------------------------- vector utilities
namespace {
constexpr int kDotBlocks = 256;

// partial[b] = sum over the grid-stride slice of block b (fixed order), then one block sums them.
__global__ void dot_partial_kernel(long long len, const double* __restrict__ x, const double* __restrict__ y,
                                   double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

__global__ void sum_kernel(int cnt, const double* __restrict__ part, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < cnt; i += 32) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) out[0] = acc;
}

struct VecList {
  const double* p[16];
  double c[16];
  int k;
};

__global__ void lincomb_kernel(long long len, VecList v, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < v.k; ++j) acc = fma(v.c[j], v.p[j][i], acc);
    out[i] = acc;
  }
}
}  // namespace

int thc_vec_dot(long long len, const double* x, const double* y, double* scratch, double* out, void* stream) {
  if (len < 0 || !x || !y || !scratch || !out) return thc::fail(nullptr, THC_EINVAL, "thc_vec_dot: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  dot_partial_kernel<<<kDotBlocks, 256, 0, s>>>(len, x, y, scratch);
  sum_kernel<<<1, 32, 0, s>>>(kDotBlocks, scratch, scratch + kDotBlocks);
  double h = 0.0;
  cudaError_t e = cudaMemcpyAsync(&h, scratch + kDotBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return thc::check_cuda(nullptr, e, "thc_vec_dot");
  *out = h;
  return THC_OK;
}

int thc_vec_lincomb(int k, const double* coeffs, const double* const* vecs, long long len, double* out, void* stream) {
  if (k < 1 || k > 16 || len < 0 || !coeffs || !vecs || !out)
    return thc::fail(nullptr, THC_EINVAL, "thc_vec_lincomb: need 1 <= k <= 16 and non-NULL arguments");
  VecList v;
  v.k = k;
  for (int j = 0; j < k; ++j) {
    if (!vecs[j]) return thc::fail(nullptr, THC_EINVAL, "thc_vec_lincomb: NULL vector");
    v.p[j] = vecs[j];
    v.c[j] = coeffs[j];
  }
  lincomb_kernel<<<(int)std::min<long long>((len + 255) / 256, 152LL * 16), 256, 0, (cudaStream_t)stream>>>(len, v,
                                                                                                           out);
  return thc::check_cuda(nullptr, cudaGetLastError(), "thc_vec_lincomb");
}

const char* thc_dyson_last_error(const thc_dyson* d) { return d ? d->err.c_str() : ""; }

void thc_dyson_destroy(thc_dyson* d) {
  if (!d) return;
  if (d->stream) cudaStreamSynchronize(d->stream);
  else cudaDeviceSynchronize();
  for (void* p : d->owned) cudaFree(p);
  delete d;
}

}  // extern "C"
