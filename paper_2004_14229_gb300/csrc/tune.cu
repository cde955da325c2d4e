// Measured launch-shape tuner of the tensor-core form (dfdm_plan_autotune):
// times candidate M2L chunk counts per level and nearfield block shapes on
// whole products, keeps the fastest, and caches the choice as one JSON line
// per plan shape.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

#include "dfdm_internal.cuh"
#include "tc.cuh"

namespace dfdm {

namespace {

struct Measured {
  double m2l[16] = {0};
  double near = 0, total = 0;
};

// One product of x with per-phase events; waits for it.
Measured timed_product(Plan &plan, const float2 *x, float2 *y, cudaStream_t st) {
  Timing &tm = plan.timing;
  const bool was_on = tm.on;
  tm.on = true;
  tm.reset();
  cudaEvent_t a = tm.next();
  DFDM_CUDA_TRY(cudaEventRecord(a, st));
  apply_tc(plan, x, y, 1, st);
  cudaEvent_t b = tm.next();
  DFDM_CUDA_TRY(cudaEventRecord(b, st));
  tm.segs.push_back(Timing::Seg{-1, a, b});
  DFDM_CUDA_TRY(cudaEventSynchronize(b));
  Measured m;
  for (const auto &s : tm.segs) {
    float ms = 0.f;
    DFDM_CUDA_TRY(cudaEventElapsedTime(&ms, s.a, s.b));
    if (s.phase == -1) m.total += ms;
    else if (s.phase == kPhNear) m.near += ms;
    else if (s.phase >= kPhM2L0 && s.phase < kPhM2L0 + 16) m.m2l[s.phase - kPhM2L0] += ms;
  }
  tm.reset();
  tm.on = was_on;
  return m;
}

void check_flag(Plan &plan, cudaStream_t st) {
  int h = 0;
  DFDM_CUDA_TRY(cudaMemcpyAsync(&h, plan.err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
  if (h != 0) throw Error{DFDM_ERR_TIMEOUT, "autotune: a device-side check failed during a timed product"};
}

// The cache line of `key`, parsed into t; false when the file has none.
bool read_cache(const char *path, const std::string &key, TcTuning &t) {
  std::ifstream f(path);
  if (!f) return false;
  const std::string want = "\"key\": \"" + key + "\"";
  std::string line;
  while (std::getline(f, line)) {
    if (line.find(want) == std::string::npos) continue;
    const size_t a = line.find("\"m2l_nsplit\": [");
    const size_t b = line.find("\"p2p\": [");
    if (a == std::string::npos || b == std::string::npos)
      throw Error{DFDM_ERR_INVALID_ARG, "autotune: cache line for this plan does not parse"};
    const char *c = line.c_str() + a + std::strlen("\"m2l_nsplit\": [");
    t.m2l_nsplit.assign(16, 0);
    for (int l = 0; l < 16; ++l) {
      char *end = nullptr;
      const long v = std::strtol(c, &end, 10);
      if (end == c || v < 0 || v > 64) throw Error{DFDM_ERR_INVALID_ARG, "autotune: bad m2l_nsplit in cache"};
      t.m2l_nsplit[l] = (int)v;
      c = end;
      while (*c == ',' || *c == ' ') ++c;
    }
    c = line.c_str() + b + std::strlen("\"p2p\": [");
    char *end = nullptr;
    const long th = std::strtol(c, &end, 10);
    c = end;
    while (*c == ',' || *c == ' ') ++c;
    const long ch = std::strtol(c, &end, 10);
    if (!(th == 0 || th == 32 || th == 64 || th == 128) || ch < 0 || ch > 16)
      throw Error{DFDM_ERR_INVALID_ARG, "autotune: bad p2p shape in cache"};
    t.p2p_threads = (int)th;
    t.p2p_chunks = (int)ch;
    return true;
  }
  return false;
}

void append_cache(const char *path, const std::string &key, const TcTuning &t, double rule_ms, double tuned_ms) {
  std::string line = "{\"key\": \"" + key + "\", \"m2l_nsplit\": [";
  for (int l = 0; l < 16; ++l) line += (l ? ", " : "") + std::to_string(l < (int)t.m2l_nsplit.size() ? t.m2l_nsplit[l] : 0);
  line += "], \"p2p\": [" + std::to_string(t.p2p_threads) + ", " + std::to_string(t.p2p_chunks) + "]";
  char buf[96];
  std::snprintf(buf, sizeof(buf), ", \"rule_ms\": %.4f, \"tuned_ms\": %.4f}\n", rule_ms, tuned_ms);
  line += buf;
  FILE *f = std::fopen(path, "a");
  if (!f) throw Error{DFDM_ERR_INVALID_ARG, std::string("autotune: cannot append to ") + path};
  const bool ok = std::fwrite(line.data(), 1, line.size(), f) == line.size();
  if (std::fclose(f) != 0 || !ok) throw Error{DFDM_ERR_INVALID_ARG, std::string("autotune: write failed: ") + path};
}

}  // namespace

void autotune_tc(Plan &plan, const float2 *x, const char *cache_path, cudaStream_t st, dfdm_tuning *out) {
  TcTuning &tune = tc_tuning(plan);
  const std::string key = tc_shape_key(plan);
  dfdm_tuning rep;
  std::memset(&rep, 0, sizeof(rep));
  TcTuning cached;
  if (cache_path && read_cache(cache_path, key, cached)) {
    // only shapes this plan would have timed itself
    for (int l = 0; l < 16; ++l) {
      const std::vector<int> c = l <= plan.depth ? tc_nsplit_candidates(plan, l) : std::vector<int>{};
      const int v = cached.m2l_nsplit[l];
      if ((c.empty() && v != 0) || (!c.empty() && std::find(c.begin(), c.end(), v) == c.end()))
        throw Error{DFDM_ERR_INVALID_ARG, "autotune: cached M2L chunk count not valid for this plan"};
    }
    const std::vector<std::pair<int, int>> pc = tc_p2p_candidates(plan);
    const std::pair<int, int> pv(cached.p2p_threads, cached.p2p_chunks);
    if ((pc.empty() && pv.first != 0) || (!pc.empty() && std::find(pc.begin(), pc.end(), pv) == pc.end()))
      throw Error{DFDM_ERR_INVALID_ARG, "autotune: cached nearfield shape not valid for this plan"};
    tune = cached;
    rep.from_cache = 1;
  } else {
    std::vector<std::vector<int>> cand(16);
    size_t passes = 1;
    for (int l = 0; l <= plan.depth && l < 16; ++l) {
      cand[l] = tc_nsplit_candidates(plan, l);
      passes = std::max(passes, cand[l].size());
    }
    const std::vector<std::pair<int, int>> pc = tc_p2p_candidates(plan);
    passes = std::max(passes, pc.size());
    float2 *y = nullptr;
    DFDM_CUDA_TRY(cudaMalloc(&y, (size_t)plan.tt.n * sizeof(float2)));
    struct Free {
      float2 *p;
      ~Free() { cudaFree(p); }
    } free_y{y};
    tune = TcTuning{};
    apply_tc(plan, x, y, 1, st);   // untimed: first touch of every table
    std::vector<std::vector<double>> lv_ms(16);
    std::vector<double> near_ms(pc.size(), 1e300);
    for (int l = 0; l < 16; ++l) lv_ms[l].assign(cand[l].size(), 1e300);
    double rule_ms = 1e300;
    for (size_t c = 0; c < passes; ++c) {
      tune.m2l_nsplit.assign(16, 0);
      for (int l = 0; l < 16; ++l)
        if (!cand[l].empty()) tune.m2l_nsplit[l] = cand[l][std::min(c, cand[l].size() - 1)];
      if (!pc.empty()) {
        tune.p2p_threads = pc[std::min(c, pc.size() - 1)].first;
        tune.p2p_chunks = pc[std::min(c, pc.size() - 1)].second;
      }
      for (int rep_i = 0; rep_i < 2; ++rep_i) {
        const Measured m = timed_product(plan, x, y, st);
        ++rep.products;
        for (int l = 0; l < 16; ++l)
          if (c < cand[l].size()) lv_ms[l][c] = std::min(lv_ms[l][c], m.m2l[l]);
        if (c < pc.size()) near_ms[c] = std::min(near_ms[c], m.near);
        if (c == 0) rule_ms = std::min(rule_ms, m.total);
      }
      check_flag(plan, st);
    }
    tune.m2l_nsplit.assign(16, 0);
    for (int l = 0; l < 16; ++l)
      if (!cand[l].empty())
        tune.m2l_nsplit[l] = cand[l][std::min_element(lv_ms[l].begin(), lv_ms[l].end()) - lv_ms[l].begin()];
    if (!pc.empty()) {
      const size_t b = std::min_element(near_ms.begin(), near_ms.end()) - near_ms.begin();
      tune.p2p_threads = pc[b].first;
      tune.p2p_chunks = pc[b].second;
    } else {
      tune.p2p_threads = tune.p2p_chunks = 0;
    }
    double tuned_ms = 1e300;
    for (int rep_i = 0; rep_i < 2; ++rep_i) {
      tuned_ms = std::min(tuned_ms, timed_product(plan, x, y, st).total);
      ++rep.products;
    }
    check_flag(plan, st);
    if (tuned_ms > rule_ms) {   // the levels interact (L2): keep the rule
      tune.m2l_nsplit.assign(16, 0);
      for (int l = 0; l < 16; ++l)
        if (!cand[l].empty()) tune.m2l_nsplit[l] = cand[l][0];
      if (!pc.empty()) {
        tune.p2p_threads = pc[0].first;
        tune.p2p_chunks = pc[0].second;
      }
    }
    rep.rule_ms = rule_ms;
    rep.tuned_ms = std::min(tuned_ms, rule_ms);
    if (cache_path) append_cache(cache_path, key, tune, rep.rule_ms, rep.tuned_ms);
  }
  for (int l = 0; l < 16; ++l) rep.m2l_nsplit[l] = l < (int)tune.m2l_nsplit.size() ? tune.m2l_nsplit[l] : 0;
  rep.p2p_threads = tune.p2p_threads;
  rep.p2p_chunks = tune.p2p_chunks;
  if (out) *out = rep;
}

}  // namespace dfdm
