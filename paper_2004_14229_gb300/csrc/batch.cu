// Batched form: many independent products (one plan each) applied together,
// their launches spread over worker streams and captured once into a CUDA
// graph that later applies replay.  Built on the public plan calls only.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "dfdm_internal.cuh"

struct dfdm_batch_s {
  std::vector<dfdm_plan> plans;
  std::vector<double> cost;            // estimated flops of one right-hand side
  std::vector<int> stream_of;          // worker stream of each problem
  std::vector<cudaStream_t> workers;
  cudaStream_t head = nullptr;         // capture origin
  std::vector<cudaEvent_t> join;       // one per worker + fork event at [0]
  cudaGraphExec_t exec = nullptr;
  std::vector<void *> key_x, key_y;    // pointers the cached graph was captured with
  int key_nrhs = 0;
  int64_t launches = 0;
};

namespace {

dfdm_status bfail(dfdm_status s, const std::string &msg) {
  dfdm::set_error(msg);
  return s;
}

void destroy_batch(dfdm_batch_s *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto e : b->join) cudaEventDestroy(e);
  for (auto s : b->workers) cudaStreamDestroy(s);
  if (b->head) cudaStreamDestroy(b->head);
  for (auto p : b->plans) dfdm_plan_destroy(p);
  delete b;
}

// Longest-processing-time-first: each problem, largest first, goes to the
// stream with the least work so far.
void schedule(dfdm_batch_s &b) {
  const int np = (int)b.plans.size(), ns = (int)b.workers.size();
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b.cost[a] > b.cost[c]; });
  std::vector<double> load(ns, 0.0);
  b.stream_of.assign(np, 0);
  for (int i : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b.stream_of[i] = s;
    load[s] += b.cost[i];
  }
}

// Captures every plan's apply on its worker stream into one graph.
dfdm_status capture(dfdm_batch_s &b, void *const *x, void *const *y, int nrhs) {
  if (b.exec) {
    cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
  }
  const int np = (int)b.plans.size(), ns = (int)b.workers.size();
  if (cudaStreamBeginCapture(b.head, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bfail(DFDM_ERR_CUDA, "cudaStreamBeginCapture failed");
  dfdm_status st = DFDM_OK;
  cudaError_t ce = cudaEventRecord(b.join[0], b.head);
  for (int w = 0; w < ns && ce == cudaSuccess; ++w) ce = cudaStreamWaitEvent(b.workers[w], b.join[0], 0);
  int64_t launches = 0;
  if (ce != cudaSuccess) st = bfail(DFDM_ERR_CUDA, "fork of the batch capture failed");
  // issue in the scheduled order (largest first on every stream)
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b.cost[a] > b.cost[c]; });
  for (int k = 0; k < np && st == DFDM_OK; ++k) {
    const int i = order[k];
    st = dfdm_apply(b.plans[i], x[i], y[i], nrhs, b.workers[b.stream_of[i]]);
    launches += b.plans[i]->p.timing.launches;
  }
  for (int w = 0; w < ns && st == DFDM_OK; ++w) {
    if (cudaEventRecord(b.join[1 + w], b.workers[w]) != cudaSuccess ||
        cudaStreamWaitEvent(b.head, b.join[1 + w], 0) != cudaSuccess)
      st = bfail(DFDM_ERR_CUDA, "join of the batch capture failed");
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b.head, &g);
  if (st == DFDM_OK && ee != cudaSuccess) st = bfail(DFDM_ERR_CUDA, "cudaStreamEndCapture failed");
  if (st == DFDM_OK && cudaGraphInstantiate(&b.exec, g, 0) != cudaSuccess) {
    b.exec = nullptr;
    st = bfail(DFDM_ERR_CUDA, "cudaGraphInstantiate failed");
  }
  if (g) cudaGraphDestroy(g);
  if (st != DFDM_OK) return st;
  b.key_x.assign(x, x + np);
  b.key_y.assign(y, y + np);
  b.key_nrhs = nrhs;
  b.launches = launches;
  return DFDM_OK;
}

}  // namespace

extern "C" {

dfdm_status dfdm_batch_create(int nprob, const dfdm_problem *probs, const dfdm_params *params, int nstreams,
                              void *stream, dfdm_batch *out) {
  if (out) *out = nullptr;
  if (!out || !probs || !params) return bfail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (nprob < 1) return bfail(DFDM_ERR_INVALID_ARG, "nprob must be >= 1");
  if (nstreams < 0 || nstreams > 64) return bfail(DFDM_ERR_INVALID_ARG, "nstreams must be in 0..64");
  if (params->n_max != 0) return bfail(DFDM_ERR_INVALID_ARG, "batched problems use uniform trees (n_max = 0)");
  dfdm_batch_s *b = new (std::nothrow) dfdm_batch_s;
  if (!b) return bfail(DFDM_ERR_OOM, "host allocation failed");
  const int ns = std::min(nstreams == 0 ? 4 : nstreams, nprob);
  for (int i = 0; i < nprob; ++i) {
    dfdm_params pi = *params;
    if (probs[i].max_depth >= 0) pi.max_depth = probs[i].max_depth;
    dfdm_plan p = nullptr;
    const dfdm_status s =
        dfdm_plan_create(probs[i].targets, probs[i].n_t, probs[i].sources, probs[i].n_s, probs[i].kappa, &pi, stream, &p);
    if (s != DFDM_OK) {
      const std::string msg = "problem " + std::to_string(i) + ": " + dfdm::last_error();
      destroy_batch(b);
      return bfail(s, msg);
    }
    b->plans.push_back(p);
    dfdm_stats st;
    dfdm_plan_stats(p, &st);
    const double n = (double)params->order * params->order * params->order;
    b->cost.push_back(8.0 * n * n * (double)st.n_coupling + 20.0 * (double)st.nf_entries +
                      16.0 * n * (double)(st.n_targets + st.n_sources));
  }
  b->workers.resize(ns, nullptr);
  b->join.resize(ns + 1, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->head, cudaStreamNonBlocking) == cudaSuccess;
  for (int w = 0; w < ns && ok; ++w) ok = cudaStreamCreateWithFlags(&b->workers[w], cudaStreamNonBlocking) == cudaSuccess;
  for (int e = 0; e <= ns && ok; ++e) ok = cudaEventCreateWithFlags(&b->join[e], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    destroy_batch(b);
    return bfail(DFDM_ERR_CUDA, "stream or event creation failed");
  }
  schedule(*b);
  *out = b;
  return DFDM_OK;
}

dfdm_status dfdm_batch_apply(dfdm_batch b, void *const *x, void *const *y, int nrhs, void *stream) {
  if (!b || !x || !y) return bfail(DFDM_ERR_INVALID_ARG, "NULL argument");
  const int np = (int)b->plans.size();
  for (int i = 0; i < np; ++i)
    if (!x[i] || !y[i]) return bfail(DFDM_ERR_INVALID_ARG, "NULL vector pointer");
  for (int i = 0; i < np; ++i)
    if (nrhs < 1 || nrhs > b->plans[i]->p.params.nrhs_max)
      return bfail(DFDM_ERR_INVALID_ARG, "nrhs must be in 1..nrhs_max");
  const bool same = b->exec && nrhs == b->key_nrhs && std::equal(x, x + np, b->key_x.begin()) &&
                    std::equal(y, y + np, b->key_y.begin());
  if (!same) {
    const dfdm_status s = capture(*b, x, y, nrhs);
    if (s != DFDM_OK) return s;
  }
  if (cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return bfail(DFDM_ERR_CUDA, "cudaGraphLaunch failed");
  return DFDM_OK;
}

dfdm_status dfdm_batch_check(dfdm_batch b, void *stream) {
  if (!b) return bfail(DFDM_ERR_INVALID_ARG, "NULL batch");
  dfdm_status first = DFDM_OK;
  for (auto p : b->plans) {
    const dfdm_status s = dfdm_plan_check(p, stream);
    if (first == DFDM_OK && s != DFDM_OK) first = s;
  }
  return first;
}

dfdm_status dfdm_batch_plan(dfdm_batch b, int i, dfdm_plan *out) {
  if (out) *out = nullptr;
  if (!b || !out) return bfail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (i < 0 || i >= (int)b->plans.size()) return bfail(DFDM_ERR_INVALID_ARG, "problem index out of range");
  *out = b->plans[i];
  return DFDM_OK;
}

dfdm_status dfdm_batch_info(dfdm_batch b, int *nstreams, int *stream_of, int64_t *launches) {
  if (!b) return bfail(DFDM_ERR_INVALID_ARG, "NULL batch");
  if (nstreams) *nstreams = (int)b->workers.size();
  if (stream_of) std::copy(b->stream_of.begin(), b->stream_of.end(), stream_of);
  if (launches) *launches = b->launches;
  return DFDM_OK;
}

dfdm_status dfdm_batch_destroy(dfdm_batch b) {
  destroy_batch(b);
  return DFDM_OK;
}

}  // extern "C"
