// FP64 evaluation of the THC second-order self-energy (Sec. II.C of
// arXiv:2404.17744): U build, per-tau SOX scheme, direct term, back-transform
// and the Galitskii-Migdal energy.  Every contraction runs in the DFMA tile
// of dfma_tile.cuh; see that file for why FP64 work is DFMA-bound on GB300.
#include <algorithm>
#include <cstdio>

#include "dfma_tile.cuh"
#include "thc_internal.cuh"

namespace thc {
namespace {

using f64::BM;
using f64::BN;
using f64::NT;
using f64::View;

constexpr double C_DIRECT = -2.0;  // closed spin loop of the bubble
constexpr double C_SOX = +1.0;     // sign reading of the SOX term on G(-tau)

inline dim3 grid_for(long long M, long long Nn, long long batch) {
  return dim3((unsigned)((M + BM - 1) / BM), (unsigned)((Nn + BN - 1) / BN), (unsigned)batch);
}

// One batched contraction; the profiler attributes 2 M Nn K batch flops to kclass.
template <bool AK, bool BK_, class LA, class LB, class Epi>
int launch_gemm(thc_ctx* ctx, int kclass, long long M, long long Nn, long long K, long long batch, const LA& a,
                const LB& b, const Epi& e, const char* what) {
  if (M <= 0 || Nn <= 0 || batch <= 0) return THC_OK;
  ProfRec rec;
  THC_TRY(prof_begin(ctx, kclass, 2.0 * M * Nn * K * batch, &rec));
  f64::gemm_kernel<AK, BK_><<<grid_for(M, Nn, batch), NT, 0, ctx->stream>>>(M, Nn, K, a, b, e);
  return prof_end(ctx, &rec, cudaGetLastError(), what);
}

// ------------------------------------------------------------------ kernels

// Fused C and D steps of the SOX scheme for one tau and one block of P:
//   C_RvP = sum_w U_Rvw G_wP          (G_wP = sum_p G_wp X_pP = Y_Pw for symmetric G)
//   D_PR  = sum_v C_RvP B_PRv
// CTA (x, y) owns R = y and 64 consecutive P of the block; it walks all v
// tiles, multiplies each C tile by the matching B entries and reduces over v
// in registers, so C is never stored.  Deterministic: no atomics.  D_PR is
// symmetric for symmetric G(+-tau), so only P <= R is computed (CTAs whose P
// all exceed R return at once) and the rest is mirrored afterwards.
__global__ void __launch_bounds__(NT) sox_cd_kernel(int n, int N, int P0, int Pcnt, const double* __restrict__ U,
                                                     const double* __restrict__ Y, const double* __restrict__ Bblk,
                                                     double* __restrict__ D) {
  __shared__ __align__(16) f64::Tiles T;
  __shared__ double red[4][BN];
  const long long R = blockIdx.y;
  const long long p0 = (long long)blockIdx.x * BN;  // local P offset in the block
  if (P0 + p0 > R) return;                          // every P of this CTA lies below the diagonal
  const f64::Lane L;
  // A(m = v, k = w) = U[R, v, w];  B(k = w, c = p) = Y[P0 + p, w]
  const View a{U + R * n * (long long)n, 0, n, 1};
  const View b{Y + (long long)P0 * n, 0, 1, n};
  double part[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long v0 = 0; v0 < n; v0 += BM) {
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    f64::mainloop<true, true>(T, a, b, 0, v0, p0, n, Pcnt, n, L, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long v = v0 + L.rm + i;
      if (v >= n) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long p = p0 + L.rn + j;
        if (p < Pcnt) part[j] = fma(acc[i][j], Bblk[(p * N + R) * n + v], part[j]);
      }
    }
  }
  // reduce over the 4 lanes along m (lane bits 3, 4), then over the 4 warps along m
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    part[j] += __shfl_xor_sync(0xffffffffu, part[j], 8);
    part[j] += __shfl_xor_sync(0xffffffffu, part[j], 16);
  }
  if (L.lm == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) red[L.wm][L.rn + j] = part[j];
  }
  __syncthreads();
  if (threadIdx.x < BN) {
    const long long p = p0 + threadIdx.x;
    if (p < Pcnt && P0 + p <= R) {
      const double s = (red[0][threadIdx.x] + red[1][threadIdx.x]) + (red[2][threadIdx.x] + red[3][threadIdx.x]);
      D[((long long)P0 + p) * N + R] = s;
    }
  }
}

// Pi (+)= G^X(tau) o G^X(-tau)^T for a batch of tau points (Pi_QS = G^X_QS(tau) G^X_SQ(-tau));
// accumulate adds the polarisation of a second spin.
__global__ void polarisation_kernel(long long N, long long batch, const double* __restrict__ GXp,
                                    const double* __restrict__ GXm, double* __restrict__ Pi, int accumulate) {
  const long long NN = N * N;
  const long long total = NN * batch;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long b = idx / NN, r = idx - b * NN;
    const long long i = r / N, j = r - i * N;
    const double p = GXp[idx] * GXm[b * NN + j * N + i];
    Pi[idx] = accumulate ? Pi[idx] + p : p;
  }
}

// D[b][P][R] = D[b][R][P] for P > R: CTA (x, y, b) writes the lower 32 x 32 tile
// (P tile y, R tile x <= y) from the upper one through shared memory.
__global__ void mirror_upper_kernel(long long N, double* __restrict__ D) {
  const long long tr = blockIdx.y, tcl = blockIdx.x;
  if (tcl > tr) return;
  __shared__ double t[32][33];
  double* Db = D + (long long)blockIdx.z * N * N;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += blockDim.y) {  // t[i][x] = D[R = 32 tcl + i][P = 32 tr + x]
    const long long R = tcl * 32 + i, P = tr * 32 + tx;
    if (R < N && P < N) t[i][tx] = Db[R * N + P];
  }
  __syncthreads();
  for (int i = ty; i < 32; i += blockDim.y) {  // D[P = 32 tr + i][R = 32 tcl + x] = t[x][i]
    const long long P = tr * 32 + i, R = tcl * 32 + tx;
    if (P < N && R < N && P > R) Db[P * N + R] = t[tx][i];
  }
}

// Epilogue of W = (V Pi) V: merged THC-space self-energy
//   M_RP = C_SOX * D_PR + cd * G^X_RP(tau) W_RP
// with cd = C_DIRECT for a restricted G (Pi of one spin, the loop's factor 2 in cd) and
// cd = -1 per spin of an unrestricted G (Pi summed over both spins).
struct MergeEpi {
  double* M;
  const double* D;    // may be null (direct term only)
  const double* GXp;
  long long N;
  double cd;
  __device__ __forceinline__ void operator()(long long b, long long r, long long p, double w) const {
    const long long o = b * N * N;
    double m = cd * GXp[o + r * N + p] * w;
    if (D) m = fma(C_SOX, D[o + r * N + p], m);  // D[p][r] = D[r][p] (mirrored): read like GXp
    M[o + r * N + p] = m;
  }
};

// Partial traces t_k = sum_ij Gb_k[i, j] S_k[j, i], one CTA per tau point.
__global__ void trace_kernel(int n, const double* __restrict__ Gb0, long long sGb, const double* __restrict__ S,
                             double* __restrict__ part) {
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
__global__ void energy_sum_kernel(int n_tau, const double* __restrict__ part, const double* __restrict__ w,
                                  double* __restrict__ out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n_tau; k += 32) acc = fma(w[k], part[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (threadIdx.x == 0) out[0] = -acc;
}

}  // namespace

size_t fp64_workspace_bytes(int n, int N, int tc, int Pb) {
  const size_t d = sizeof(double);
  const size_t NN = (size_t)N * N, Nn = (size_t)N * n;
  return d * ((size_t)tc * (2 * Nn + 4 * NN + Nn) + (size_t)Pb * ((size_t)n * n + Nn));
}

// U_Pqs = sum_Q V_PQ X_qQ X_sQ (Eq. U_contraction), the Khatri-Rao operand generated in the loader.
int fp64_build_U(thc_ctx* ctx) {
  const long long n = ctx->n, N = ctx->N;
  const View a{ctx->V, 0, N, 1};                 // A(m = P, k = Q) = V[P, Q]
  const f64::KhatriRao b{ctx->X, ctx->n, ctx->N};  // B(k = Q, c = q n + s)
  const f64::StoreEpi e{ctx->U, 0, n * n, 1, 1.0};
  return launch_gemm<true, true>(ctx, K_UBUILD, N, n * n, N, 1, a, b, e, "U build");
}

namespace {

// Views of G(tau_k) and G(beta - tau_k) for the tau points c0 .. of one chunk.
struct SpinIn {
  View g, gb;
};
SpinIn spin_views(thc_ctx* ctx, const double* G_tau, const double* G_bmt, long long c0) {
  const long long n = ctx->n, nn = n * n, nt = ctx->n_tau;
  SpinIn v;
  v.g = View{G_tau + c0 * nn, nn, n, 1};
  v.gb = G_bmt ? View{G_bmt + c0 * nn, nn, n, 1} : View{G_tau + (nt - 1 - c0) * nn, -nn, n, 1};
  return v;
}

// Y = X^T G(tau) (always), and with the direct term Ym = X^T G(-tau), G^X(+-tau)
// (G^X(-tau) only when need_minus) for one spin and chunk.
int fp64_project(thc_ctx* ctx, const SpinIn& in, long long tc, bool dir, bool need_minus) {
  const long long n = ctx->n, N = ctx->N, NN = N * N, Nn = N * n;
  // Y_Rq = sum_u X_uR G_uq(tau): computed as (m = q, c = R), A(q, u) = G[u, q], B(u, R) = X[u, R]
  const View b{ctx->X, 0, N, 1};
  THC_TRY(launch_gemm<false, false>(ctx, K_PROJECT, n, N, n, tc, View{in.g.p, in.g.sb, 1, n}, b,
                                    f64::StoreEpi{ctx->Y, Nn, 1, n, 1.0}, "Y"));
  if (!dir) return THC_OK;
  if (need_minus)  // Ym = X^T G(-tau) = -X^T G(beta - tau)
    THC_TRY(launch_gemm<false, false>(ctx, K_PROJECT, n, N, n, tc, View{in.gb.p, in.gb.sb, 1, n}, b,
                                      f64::StoreEpi{ctx->Ym, Nn, 1, n, -1.0}, "Ym"));
  // G^X(+-tau) = Y(+-) X : (m = P, c = R), A(P, q) = Y[P, q], B(q, R) = X[q, R]
  THC_TRY(launch_gemm<true, false>(ctx, K_PROJECT, N, N, n, tc, View{ctx->Y, Nn, n, 1}, b,
                                   f64::StoreEpi{ctx->GXp, NN, N, 1, 1.0}, "GX+"));
  if (need_minus)
    THC_TRY(launch_gemm<true, false>(ctx, K_PROJECT, N, N, n, tc, View{ctx->Ym, Nn, n, 1}, b,
                                     f64::StoreEpi{ctx->GXm, NN, N, 1, 1.0}, "GX-"));
  return THC_OK;
}

int fp64_polarisation(thc_ctx* ctx, long long tc, bool accumulate) {
  const long long N = ctx->N, NN = N * N;
  const long long total = NN * tc;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_POLARISATION, 0.0, &rec));
  polarisation_kernel<<<blocks, 256, 0, ctx->stream>>>(N, tc, ctx->GXp, ctx->GXm, ctx->Pi, accumulate ? 1 : 0);
  return prof_end(ctx, &rec, cudaGetLastError(), "polarisation");
}

// D_PR (all tau of the chunk) of the SOX scheme from Y (this spin's projection) and G(-tau).
int fp64_sox(thc_ctx* ctx, const SpinIn& in, long long tc) {
  const long long n = ctx->n, N = ctx->N, nn = n * n, NN = N * N, Nn = N * n;
  for (long long k = 0; k < tc; ++k) {
    const double* Gb = in.gb.p + k * in.gb.sb;  // G(beta - tau_k)
    const double* Yk = ctx->Y + k * Nn;
    double* Dk = ctx->D + k * NN;
    for (long long P0 = 0; P0 < N; P0 += ctx->Pb) {
      const long long Pc = std::min<long long>(ctx->Pb, N - P0);
      // A_Pqv = sum_s U_Pqs G_sv(-tau) = -sum_s U_Pqs G_sv(beta - tau):
      // (m = v, c = (P, q)), A(v, s) = Gb[s, v], B(s, (P, q)) = U[P0 + P, q, s]
      THC_TRY(launch_gemm<false, true>(ctx, K_SOX_A, n, Pc * n, n, 1, View{Gb, 0, 1, n},
                                       View{ctx->U + P0 * nn, 0, 1, n}, f64::StoreEpi{ctx->Ablk, 0, 1, n, -1.0},
                                       "A"));
      // B_PRv = sum_q A_Pqv G_Rq (batched over P): (m = v, c = R), A(v, q) = A[P, q, v], B(q, R) = Y[R, q];
      // only R >= P is used (D is symmetric): column tiles wholly left of P are skipped
      double bflops = 0.0, cdflops = 0.0;  // multiply-adds the kernels carry out, x 2
      for (long long b = 0; b < Pc; ++b) bflops += 2.0 * n * n * (N - (P0 + b) / BN * BN);
      for (long long p0 = 0; p0 < Pc; p0 += BN)
        if (P0 + p0 < N) cdflops += (2.0 * nn + 2.0 * n) * std::min<long long>(BN, Pc - p0) * (N - (P0 + p0));
      {
        ProfRec rec;
        THC_TRY(prof_begin(ctx, K_SOX_B, bflops, &rec));
        f64::gemm_kernel<false, true><<<grid_for(n, N, Pc), NT, 0, ctx->stream>>>(
            n, N, n, View{ctx->Ablk, nn, 1, n}, View{Yk, 0, 1, n}, f64::TriStoreEpi{ctx->Bblk, Nn, 1, n, 1.0, P0});
        THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "B"));
      }
      // C and D fused, P <= R
      ProfRec rec;
      THC_TRY(prof_begin(ctx, K_SOX_CD, cdflops, &rec));
      sox_cd_kernel<<<dim3((unsigned)((Pc + BN - 1) / BN), (unsigned)N), NT, 0, ctx->stream>>>(
          (int)n, (int)N, (int)P0, (int)Pc, ctx->U, Yk, ctx->Bblk, Dk);
      THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "C/D"));
    }
  }
  return launch_mirror_upper(ctx, ctx->D, N, tc);
}

// Sigma = X M X^T for the tau points of the chunk, M_RP = M[R][P] in the Pi buffer (merged)
// or, without the direct term, M_RP = C_SOX D[P][R].
int fp64_back(thc_ctx* ctx, long long tc, bool merged, double* Sigma_chunk) {
  const long long n = ctx->n, N = ctx->N, nn = n * n, NN = N * N, Nn = N * n;
  // T2 = M X^T : (m = R, c = r), A(R, P) = M[R, P], B(P, r) = X[r, P]
  if (merged)
    THC_TRY(launch_gemm<true, true>(ctx, K_BACK, N, n, N, tc, View{ctx->Pi, NN, N, 1}, View{ctx->X, 0, 1, N},
                                    f64::StoreEpi{ctx->T2, Nn, n, 1, 1.0}, "M X^T"));
  else
    THC_TRY(launch_gemm<false, true>(ctx, K_BACK, N, n, N, tc, View{ctx->D, NN, 1, N}, View{ctx->X, 0, 1, N},
                                     f64::StoreEpi{ctx->T2, Nn, n, 1, C_SOX}, "M X^T"));
  // Sigma = X T2 : (m = t, c = r), A(t, R) = X[t, R], B(R, r) = T2[R, r]
  return launch_gemm<true, false>(ctx, K_BACK, n, n, N, tc, View{ctx->X, 0, N, 1}, View{ctx->T2, Nn, n, 1},
                                  f64::StoreEpi{Sigma_chunk, nn, n, 1, 1.0}, "X T2");
}

// M = C_SOX D^T + cd G^X o (T V) with T = V Pi already in the GXm buffer (direct term), or
// M = C_SOX D^T alone; then the back-transform.
int fp64_merge_back(thc_ctx* ctx, long long tc, bool sox, bool dir, double cd, double* Sigma_chunk) {
  const long long N = ctx->N, NN = N * N;
  if (dir)
    THC_TRY(launch_gemm<true, false>(ctx, K_DIRECT_W, N, N, N, tc, View{ctx->GXm, NN, N, 1}, View{ctx->V, 0, N, 1},
                                     MergeEpi{ctx->Pi, sox ? ctx->D : nullptr, ctx->GXp, N, cd}, "W"));
  return fp64_back(ctx, tc, dir, Sigma_chunk);
}

// Screened direct term (THC_GW) with or without SOX, restricted (nspin 1) or unrestricted
// (nspin 2): the bubble of every tau point first (the bosonic transform couples them;
// unrestricted, spin b and then spin a added), then W~(tau), then per chunk and spin SOX,
// the merge M = C_SOX D^T - G^X_s o W~ and the back-transform.
int fp64_eval_gw(thc_ctx* ctx, int nspin, const double* const* G_tau, const double* const* G_bmt,
                 double* const* Sigma) {
  const long long n = ctx->n, nt = ctx->n_tau, nn = n * n;
  const bool sox = ctx->terms & THC_SOX;
  if (!ctx->gw_nw) return fail(ctx, THC_EINVAL, "THC_GW needs the bosonic transforms (thc_sigma_set_bosonic)");
  for (long long c0 = 0; c0 < nt; c0 += ctx->tc) {
    const long long tc = std::min<long long>(ctx->tc, nt - c0);
    for (int s = nspin - 1; s >= 0; --s) {
      THC_TRY(fp64_project(ctx, spin_views(ctx, G_tau[s], G_bmt[s], c0), tc, true, true));
      THC_TRY(gw_store_bubble(ctx, c0, tc, nspin, s));
    }
  }
  THC_TRY(gw_screen(ctx));
  for (long long c0 = 0; c0 < nt; c0 += ctx->tc) {
    const long long tc = std::min<long long>(ctx->tc, nt - c0);
    for (int s = 0; s < nspin; ++s) {
      const SpinIn in = spin_views(ctx, G_tau[s], G_bmt[s], c0);
      if (sox) {
        THC_TRY(fp64_project(ctx, in, tc, false, false));  // Y for the SOX scheme
        THC_TRY(fp64_sox(ctx, in, tc));
      }
      THC_TRY(gw_merge(ctx, c0, tc, sox ? ctx->D : nullptr, ctx->Pi, s));
      THC_TRY(fp64_back(ctx, tc, true, Sigma[s] + c0 * nn));
    }
  }
  return THC_OK;
}

}  // namespace

// Restricted (nspin = 1: one per-spin G, direct factor C_DIRECT) or unrestricted
// (nspin = 2: G of spin a and b, polarisation summed over both spins, direct factor -1
// per spin, SOX within each spin); with THC_GW the screened evaluation above.  Order per chunk, unrestricted: project b and form
// Pi_b; project a and add Pi_a; T = V Pi; SOX a, merge a, back-transform a; project b
// again (Y, G^X(tau)), SOX b, merge b, back-transform b.
int fp64_eval_spins(thc_ctx* ctx, int nspin, const double* const* G_tau, const double* const* G_bmt,
                    double* const* Sigma) {
  if (ctx->terms & THC_GW) return fp64_eval_gw(ctx, nspin, G_tau, G_bmt, Sigma);
  const long long n = ctx->n, N = ctx->N, nt = ctx->n_tau, nn = n * n, NN = N * N;
  const bool sox = ctx->terms & THC_SOX, dir = ctx->terms & THC_DIRECT;
  const double cd = nspin == 1 ? C_DIRECT : -1.0;
  for (long long c0 = 0; c0 < nt; c0 += ctx->tc) {
    const long long tc = std::min<long long>(ctx->tc, nt - c0);
    SpinIn in[2];
    for (int s = 0; s < nspin; ++s) in[s] = spin_views(ctx, G_tau[s], G_bmt[s], c0);
    if (nspin == 2 && dir) {  // Pi of spin b first
      THC_TRY(fp64_project(ctx, in[1], tc, true, true));
      THC_TRY(fp64_polarisation(ctx, tc, false));
    }
    THC_TRY(fp64_project(ctx, in[0], tc, dir, true));
    if (dir) {
      THC_TRY(fp64_polarisation(ctx, tc, nspin == 2));
      // T = V Pi -> GXm buffer (G^X(-tau) is not needed after Pi)
      THC_TRY(launch_gemm<true, false>(ctx, K_DIRECT_VPI, N, N, N, tc, View{ctx->V, 0, N, 1}, View{ctx->Pi, NN, N, 1},
                                       f64::StoreEpi{ctx->GXm, NN, N, 1, 1.0}, "V Pi"));
    }
    for (int s = 0; s < nspin; ++s) {
      if (s == 1) THC_TRY(fp64_project(ctx, in[1], tc, dir, false));  // Y and G^X(tau) of spin b
      if (sox) THC_TRY(fp64_sox(ctx, in[s], tc));
      THC_TRY(fp64_merge_back(ctx, tc, sox, dir, cd, Sigma[s] + c0 * nn));
    }
  }
  return THC_OK;
}

int fp64_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, double* Sigma) {
  return fp64_eval_spins(ctx, 1, &G_tau, &G_bmt, &Sigma);
}

int energy_eval(thc_ctx* ctx, const double* G_tau, const double* G_bmt, const double* Sigma,
                const double* w_host, double* E) {
  const long long n = ctx->n, nt = ctx->n_tau, nn = n * n;
  const double* gb0 = G_bmt ? G_bmt : G_tau + (nt - 1) * nn;
  const long long sgb = G_bmt ? nn : -nn;
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(ctx->e_w, w_host, sizeof(double) * nt, cudaMemcpyHostToDevice, ctx->stream),
                     "copy weights"));
  ProfRec rec;
  THC_TRY(prof_begin(ctx, K_ENERGY, 0.0, &rec));
  trace_kernel<<<(unsigned)nt, 256, 0, ctx->stream>>>((int)n, gb0, sgb, Sigma, ctx->e_part);
  THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "trace"));
  THC_TRY(prof_begin(ctx, K_ENERGY, 0.0, &rec));
  energy_sum_kernel<<<1, 32, 0, ctx->stream>>>((int)nt, ctx->e_part, ctx->e_w, ctx->e_out);
  THC_TRY(prof_end(ctx, &rec, cudaGetLastError(), "energy sum"));
  THC_TRY(check_cuda(ctx, cudaMemcpyAsync(E, ctx->e_out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                     "copy energy"));
  return check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "energy sync");
}

int launch_mirror_upper(thc_ctx* ctx, double* D, long long N, long long batch) {
  if (N <= 1 || batch <= 0) return THC_OK;
  const unsigned t = (unsigned)((N + 31) / 32);
  mirror_upper_kernel<<<dim3(t, t, (unsigned)batch), dim3(32, 8, 1), 0, ctx->stream>>>(N, D);
  return check_cuda(ctx, cudaGetLastError(), "mirror D");
}

}  // namespace thc
