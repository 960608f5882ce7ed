// Batched self-energy evaluation over many molecules of uneven size.
//
// Each molecule has its own context (U, blocking, workspace) bound to one of
// a few worker streams, so small molecules that cannot fill the GPU run
// concurrently.  The first evaluation runs every molecule once outside
// capture (with the tensor-core autotuner on, when requested) and then
// captures the fork / per-molecule work / join into one CUDA graph; later
// evaluations with the same buffers replay the graph in a single launch.
#include <algorithm>
#include <string>
#include <vector>

#include "thc_internal.cuh"
#include "thc_batch.h"

struct thc_batch {
  int n_mol = 0, n_tau = 0, precision = THC_FP64, tune = 0;
  cudaStream_t main = nullptr;        // the caller's stream: graph launches are ordered on it
  cudaStream_t cap = nullptr;         // private root stream of the warm-up and the capture
  cudaEvent_t ready = nullptr;        // caller's work before the first evaluation
  std::vector<cudaStream_t> workers;
  std::vector<thc_ctx*> ctx;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const double*> g_key;
  std::vector<double*> s_key;
  size_t graph_nodes = 0;
  long long launches = 0;
  std::string err;
};

namespace {

int bfail(thc_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return thc::fail(nullptr, code, msg);
}

int bcheck(thc_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return THC_OK;
  return bfail(b, e == cudaErrorMemoryAllocation ? THC_ENOMEM : THC_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

void drop_graph(thc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// fork from the root stream, every molecule on its worker, join back
int enqueue_all(thc_batch* b, const double* const* G, double* const* S) {
  THC_TRY(bcheck(b, cudaEventRecord(b->fork, b->cap), "fork"));
  for (cudaStream_t w : b->workers) THC_TRY(bcheck(b, cudaStreamWaitEvent(w, b->fork, 0), "fork wait"));
  for (int i = 0; i < b->n_mol; ++i) {
    thc_ctx* c = b->ctx[i];
    const int rc = (c->precision == THC_FP64) ? thc::fp64_eval(c, G[i], nullptr, S[i]) : thc::split_eval(c, G[i], nullptr, S[i]);
    if (rc != THC_OK) return bfail(b, rc, "molecule " + std::to_string(i) + ": " + c->err);
  }
  for (size_t w = 0; w < b->workers.size(); ++w) {
    THC_TRY(bcheck(b, cudaEventRecord(b->join[w], b->workers[w]), "join"));
    THC_TRY(bcheck(b, cudaStreamWaitEvent(b->cap, b->join[w], 0), "join wait"));
  }
  return THC_OK;
}

}  // namespace

extern "C" {

int thc_batch_init(thc_batch** out, int n_mol, const int* n_ao, const int* n_thc, int n_tau, double beta,
                   const double* const* X, const double* const* V, const double* tau, int precision, int n_streams,
                   unsigned long long budget_per_molecule, int tune, void* stream) {
  if (!out) return thc::fail(nullptr, THC_EINVAL, "thc_batch_init: NULL out-pointer");
  *out = nullptr;
  if (n_mol < 1 || !n_ao || !n_thc || !X || !V || !tau || n_streams < 1 || n_streams > 64)
    return thc::fail(nullptr, THC_EINVAL, "thc_batch_init: bad arguments (1 <= n_streams <= 64)");
  thc_batch* b = new (std::nothrow) thc_batch();
  if (!b) return thc::fail(nullptr, THC_ENOMEM, "thc_batch_init: host allocation");
  b->n_mol = n_mol;
  b->n_tau = n_tau;
  b->precision = precision;
  b->tune = tune;
  b->main = (cudaStream_t)stream;
  int rc = bcheck(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  if (rc == THC_OK) rc = bcheck(b, cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming), "event");
  if (rc == THC_OK) rc = bcheck(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "capture stream");
  const int ns = std::min(n_streams, n_mol);
  for (int w = 0; w < ns && rc == THC_OK; ++w) {
    cudaStream_t s;
    rc = bcheck(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "worker stream");
    if (rc == THC_OK) b->workers.push_back(s);
    cudaEvent_t e;
    if (rc == THC_OK) rc = bcheck(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    if (rc == THC_OK) b->join.push_back(e);
  }
  // per-molecule workspace: explicit, or an equal share of a quarter of the free memory
  size_t budget = (size_t)budget_per_molecule;
  if (rc == THC_OK && budget == 0) {
    size_t free_b = 0, total_b = 0;
    rc = bcheck(b, cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    budget = std::max<size_t>(free_b / 4 / (size_t)n_mol, (size_t)64 << 20);
  }
  for (int i = 0; i < n_mol && rc == THC_OK; ++i) {
    thc_ctx* c = nullptr;
    rc = thc::ctx_create(&c, n_ao[i], n_thc[i], n_tau, beta, X[i], V[i], tau, precision, THC_DIRECT | THC_SOX,
                         b->workers[i % ns], budget);
    if (rc != THC_OK) {
      rc = bfail(b, rc, "molecule " + std::to_string(i) + ": " + thc_last_error(nullptr));
      break;
    }
    if (!c->mirrored) {
      thc::ctx_destroy(c);
      rc = bfail(b, THC_EINVAL, "thc_batch_init: the tau grid must be mirror-symmetric");
      break;
    }
    b->ctx.push_back(c);
  }
  if (rc == THC_OK) rc = bcheck(b, cudaDeviceSynchronize(), "batch init sync");
  if (rc != THC_OK) {
    thc_batch_destroy(b);
    return rc;
  }
  *out = b;
  return THC_OK;
}

int thc_batch_eval(thc_batch* b, const double* const* G_tau, double* const* Sigma_tau) {
  if (!b || !G_tau || !Sigma_tau) return thc::fail(nullptr, THC_EINVAL, "thc_batch_eval: NULL argument");
  for (int i = 0; i < b->n_mol; ++i)
    if (!G_tau[i] || !Sigma_tau[i] || G_tau[i] == Sigma_tau[i])
      return bfail(b, THC_EINVAL, "thc_batch_eval: NULL or aliased buffer of molecule " + std::to_string(i));
  bool same = b->exec && (int)b->g_key.size() == b->n_mol;
  for (int i = 0; same && i < b->n_mol; ++i) same = b->g_key[i] == G_tau[i] && b->s_key[i] == Sigma_tau[i];
  if (!same) {
    drop_graph(b);
    // warm-up outside capture, after the caller's queued work: sets kernel attributes and,
    // when asked, tunes the tile widths
    THC_TRY(bcheck(b, cudaEventRecord(b->ready, b->main), "ready"));
    THC_TRY(bcheck(b, cudaStreamWaitEvent(b->cap, b->ready, 0), "ready wait"));
    for (thc_ctx* c : b->ctx) c->tuning = b->tune != 0;
    int rc = enqueue_all(b, G_tau, Sigma_tau);
    for (thc_ctx* c : b->ctx) c->tuning = false;
    THC_TRY(rc);
    THC_TRY(bcheck(b, cudaStreamSynchronize(b->cap), "warm-up sync"));
    long long before = 0;
    for (thc_ctx* c : b->ctx) before += c->launch_count;
    THC_TRY(bcheck(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture"));
    rc = enqueue_all(b, G_tau, Sigma_tau);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
    if (rc != THC_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    THC_TRY(bcheck(b, ec, "end capture"));
    b->graph = g;
    THC_TRY(bcheck(b, cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate"));
    size_t nodes = 0;
    THC_TRY(bcheck(b, cudaGraphGetNodes(b->graph, nullptr, &nodes), "graph nodes"));
    b->graph_nodes = nodes;
    long long after = 0;
    for (thc_ctx* c : b->ctx) after += c->launch_count;
    b->launches = after - before;
    b->g_key.assign(G_tau, G_tau + b->n_mol);
    b->s_key.assign(Sigma_tau, Sigma_tau + b->n_mol);
  }
  return bcheck(b, cudaGraphLaunch(b->exec, b->main), "graph launch");
}

int thc_batch_graph_info(const thc_batch* b, long long* kernel_launches, long long* graph_nodes) {
  if (!b) return thc::fail(nullptr, THC_EINVAL, "thc_batch_graph_info: NULL batch");
  if (kernel_launches) *kernel_launches = b->launches;
  if (graph_nodes) *graph_nodes = (long long)b->graph_nodes;
  return THC_OK;
}

double thc_batch_flops(const thc_batch* b) {
  if (!b) return 0.0;
  double f = 0.0;
  for (const thc_ctx* c : b->ctx) f += thc_sigma_flops(c, nullptr);
  return f;
}

const char* thc_batch_last_error(const thc_batch* b) { return b ? b->err.c_str() : ""; }

void thc_batch_destroy(thc_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  drop_graph(b);
  for (thc_ctx* c : b->ctx) thc::ctx_destroy(c);
  for (cudaStream_t s : b->workers) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ready) cudaEventDestroy(b->ready);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // extern "C"
