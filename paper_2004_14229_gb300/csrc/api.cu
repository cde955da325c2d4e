// C ABI of the library (include/dfdm.h): validation, plan assembly, apply
// dispatch, counters and exports.
#include <cmath>
#include <cstring>
#include <new>

#include "dfdm_internal.cuh"
#include "tc.cuh"

namespace dfdm {

namespace {
thread_local std::string g_last_error = "no error";
}

void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error() { return g_last_error.c_str(); }

void Plan::free_all() {
  destroy_tc(*this);
  timing.destroy();
  for (auto &b : owned) cudaFree(b.ptr);
  owned.clear();
  if (x_stage) cudaFreeHost(x_stage);
  if (y_stage) cudaFreeHost(y_stage);
  x_stage = y_stage = nullptr;
  device_bytes = 0;
}

namespace {

dfdm_status fail(dfdm_status s, const std::string &msg) {
  set_error(msg);
  return s;
}

template <typename F>
dfdm_status guarded(F &&f) {
  try {
    return f();
  } catch (const Error &e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return DFDM_ERR_OOM;
  } catch (const std::exception &e) {
    set_error(e.what());
    return DFDM_ERR_CUDA;
  }
}

bool finite_points(const double *p, int64_t n) {
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Smallest power-of-two cube on a dyadic corner holding both point sets.
void bounding_root(const double *t, int64_t nt, const double *s, int64_t ns,
                   double lo[3], double &side) {
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < nt; ++i)
    for (int a = 0; a < 3; ++a) {
      mn[a] = std::fmin(mn[a], t[3 * i + a]);
      mx[a] = std::fmax(mx[a], t[3 * i + a]);
    }
  for (int64_t i = 0; i < ns; ++i)
    for (int a = 0; a < 3; ++a) {
      mn[a] = std::fmin(mn[a], s[3 * i + a]);
      mx[a] = std::fmax(mx[a], s[3 * i + a]);
    }
  double ext = 0;
  for (int a = 0; a < 3; ++a) ext = std::fmax(ext, mx[a] - mn[a]);
  int e = (ext > 0) ? (int)std::ceil(std::log2(ext)) : -20;
  for (;;) {
    side = std::ldexp(1.0, e);
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::floor(mn[a] / side) * side;
      if (lo[a] + side < mx[a]) ok = false;
    }
    if (ok) break;
    ++e;
  }
}

}  // namespace
}  // namespace dfdm

using namespace dfdm;


extern "C" {

dfdm_status dfdm_params_default(dfdm_params *p) {
  if (!p) return fail(DFDM_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->order = 5;
  p->max_depth = 6;
  p->n_max = 0;
  p->eta2 = 5.0;
  p->l_hf = -2;
  p->root_mode = 0;
  p->root_lo[0] = p->root_lo[1] = p->root_lo[2] = 0.0;
  p->root_side = 1.0;
  p->precision = DFDM_FP64;
  p->nrhs_max = 1;
  return DFDM_OK;
}

dfdm_status dfdm_plan_create(const double *targets, int64_t n_t,
                             const double *sources, int64_t n_s, double kappa,
                             const dfdm_params *params, void *stream,
                             dfdm_plan *out) {
  if (out) *out = nullptr;
  if (!out || !params) return fail(DFDM_ERR_INVALID_ARG, "out or params is NULL");
  if (!targets || !sources) return fail(DFDM_ERR_INVALID_ARG, "point pointer is NULL");
  if (n_t < 1 || n_s < 1) return fail(DFDM_ERR_INVALID_ARG, "point counts must be >= 1");
  if (n_t > (int64_t)1 << 30 || n_s > (int64_t)1 << 30)
    return fail(DFDM_ERR_INVALID_ARG, "at most 2^30 points per set");
  if (!(kappa > 0) || !std::isfinite(kappa)) return fail(DFDM_ERR_INVALID_ARG, "kappa must be finite and > 0");
  const dfdm_params &pr = *params;
  if (pr.order < 2 || pr.order > kMaxOrder) return fail(DFDM_ERR_INVALID_ARG, "order must be in 2..10");
  if (pr.max_depth < 0 || pr.max_depth > kMaxDepth) return fail(DFDM_ERR_INVALID_ARG, "max_depth must be in 0..10");
  if (pr.n_max < 0) return fail(DFDM_ERR_INVALID_ARG, "n_max must be >= 0");
  if (!(pr.eta2 > 0) || !std::isfinite(pr.eta2)) return fail(DFDM_ERR_INVALID_ARG, "eta2 must be > 0");
  if (pr.l_hf < -2) return fail(DFDM_ERR_INVALID_ARG, "l_hf must be >= -2");
  if (pr.nrhs_max < 1) return fail(DFDM_ERR_INVALID_ARG, "nrhs_max must be >= 1");
  if (pr.precision != DFDM_FP64 && pr.precision != DFDM_TC_FP16X3)
    return fail(DFDM_ERR_INVALID_ARG, "unknown precision");
  if (pr.precision == DFDM_TC_FP16X3 && pr.order > 6)
    return fail(DFDM_ERR_UNSUPPORTED, "the tensor-core form supports orders 2..6");
  if (pr.root_mode != 0 && pr.root_mode != 1) return fail(DFDM_ERR_INVALID_ARG, "root_mode must be 0 or 1");
  if (!finite_points(targets, n_t) || !finite_points(sources, n_s))
    return fail(DFDM_ERR_INVALID_ARG, "coordinates must be finite");
  dfdm_plan_s *h = new (std::nothrow) dfdm_plan_s;
  if (!h) return fail(DFDM_ERR_OOM, "host allocation failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dfdm_status s = guarded([&]() -> dfdm_status {
    Plan &plan = h->p;
    plan.params = pr;
    plan.kappa = kappa;
    plan.order = pr.order;
    plan.n = pr.order * pr.order * pr.order;
    if (pr.root_mode == 0) {
      if (!(pr.root_side > 0) || !std::isfinite(pr.root_side))
        throw Error{DFDM_ERR_INVALID_ARG, "root_side must be finite and > 0"};
      for (int a = 0; a < 3; ++a) {
        plan.root_lo[a] = pr.root_lo[a];
        if (!std::isfinite(pr.root_lo[a])) throw Error{DFDM_ERR_INVALID_ARG, "root_lo must be finite"};
      }
      plan.root_side = pr.root_side;
      for (int64_t i = 0; i < n_t; ++i)
        for (int a = 0; a < 3; ++a)
          if (targets[3 * i + a] < plan.root_lo[a] || targets[3 * i + a] > plan.root_lo[a] + plan.root_side)
            throw Error{DFDM_ERR_INVALID_ARG, "a target lies outside the root cube"};
      for (int64_t i = 0; i < n_s; ++i)
        for (int a = 0; a < 3; ++a)
          if (sources[3 * i + a] < plan.root_lo[a] || sources[3 * i + a] > plan.root_lo[a] + plan.root_side)
            throw Error{DFDM_ERR_INVALID_ARG, "a source lies outside the root cube"};
    } else {
      bounding_root(targets, n_t, sources, n_s, plan.root_lo, plan.root_side);
    }
    build_tree(plan, plan.tt, targets, n_t, st);
    build_tree(plan, plan.ts, sources, n_s, st);
    if (plan.tt.depth != plan.ts.depth)
      throw Error{DFDM_ERR_UNSUPPORTED, "target and source trees have different depths"};
    plan.depth = plan.tt.depth;
    plan.l_hf = (pr.l_hf == -2) ? default_l_hf(kappa, plan.root_side, plan.depth) : pr.l_hf;
    if (plan.l_hf > plan.depth) plan.l_hf = plan.depth;
    build_levels(plan);
    build_operators_fp64(plan, st);
    count_pairs(plan, st);
    const int p = plan.depth;
    // moments / locals / scratch
    plan.mom.assign(p + 1, nullptr);
    plan.loc.assign(p + 1, nullptr);
    if (pr.precision == DFDM_FP64) {
      for (int l = plan.min_level; l <= p; ++l) {
        const size_t cnt = plan.levels[l].slot_dir.size() * ((size_t)1 << (3 * l)) * plan.n;
        plan.mom[l] = plan.alloc<double2>(cnt);
        plan.loc[l] = plan.alloc<double2>(cnt);
      }
      plan.ysorted = plan.alloc<double2>(plan.tt.n);
    } else {
      build_tc(plan, st);
    }
    const size_t elem = (pr.precision == DFDM_FP64) ? 16 : 8;
    plan.stage_bytes = (size_t)pr.nrhs_max * (size_t)std::max(n_t, n_s) * elem;
    plan.x_dev_stage = plan.alloc<char>(plan.stage_bytes);
    plan.y_dev_stage = plan.alloc<char>(plan.stage_bytes);
    DFDM_CUDA_TRY(cudaMallocHost(&plan.x_stage, plan.stage_bytes));
    DFDM_CUDA_TRY(cudaMallocHost(&plan.y_stage, plan.stage_bytes));
    plan.err_flag = plan.alloc<int>(1);
    DFDM_CUDA_TRY(cudaMemsetAsync(plan.err_flag, 0, sizeof(int), st));
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    // counters
    dfdm_stats &S = plan.stats;
    S.n_targets = n_t;
    S.n_sources = n_s;
    S.depth = p;
    S.l_hf = plan.l_hf;
    S.n_stored_coupling = plan.n_ops;
    S.n_leaves_t = plan.tt.nleaves;
    S.n_leaves_s = plan.ts.nleaves;
    for (int l = 0; l <= p && l < 16; ++l) {
      S.level_dirs[l] = (int32_t)plan.levels[l].slot_dir.size();
      S.level_coupling[l] = plan.levels[l].n_coupling;
      S.level_offsets[l] = (int32_t)plan.levels[l].op_dir.size();
    }
    S.device_bytes = plan.device_bytes;
    return DFDM_OK;
  });
  if (s != DFDM_OK) {
    h->p.free_all();
    delete h;
    return s;
  }
  *out = h;
  return DFDM_OK;
}

dfdm_status dfdm_apply(dfdm_plan plan, const void *x, void *y, int nrhs, void *stream) {
  if (!plan || !x || !y) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (nrhs < 1 || nrhs > plan->p.params.nrhs_max)
    return fail(DFDM_ERR_INVALID_ARG, "nrhs must be in 1..nrhs_max");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> dfdm_status {
    Timing &tm = plan->p.timing;
    tm.launches = 0;
    if (!tm.on) tm.reset();   // with timing on, segments accumulate until read
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (tm.on) {
      t0 = tm.next();
      DFDM_CUDA_TRY(cudaEventRecord(t0, st));
    }
    if (plan->p.params.precision == DFDM_FP64)
      apply_fp64(plan->p, static_cast<const double2 *>(x), static_cast<double2 *>(y), nrhs, st);
    else
      apply_tc(plan->p, static_cast<const float2 *>(x), static_cast<float2 *>(y), nrhs, st);
    if (tm.on) {
      t1 = tm.next();
      DFDM_CUDA_TRY(cudaEventRecord(t1, st));
      tm.segs.push_back(Timing::Seg{-1, t0, t1});
      tm.acc_launches += tm.launches;
      ++tm.applies;
      tm.valid = true;
    }
    return DFDM_OK;
  });
}

dfdm_status dfdm_plan_set_timing(dfdm_plan plan, int enable) {
  if (!plan) return fail(DFDM_ERR_INVALID_ARG, "NULL plan");
  plan->p.timing.on = enable != 0;
  plan->p.timing.reset();
  return DFDM_OK;
}

dfdm_status dfdm_plan_autotune(dfdm_plan plan, const void *x, const char *cache_path, void *stream,
                               dfdm_tuning *out) {
  if (!plan || !x) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (plan->p.params.precision != DFDM_TC_FP16X3)
    return fail(DFDM_ERR_INVALID_ARG, "autotune applies to the tensor-core form only");
  return guarded([&]() -> dfdm_status {
    autotune_tc(plan->p, static_cast<const float2 *>(x), cache_path, static_cast<cudaStream_t>(stream), out);
    return DFDM_OK;
  });
}

dfdm_status dfdm_plan_timing(dfdm_plan plan, dfdm_timing *t) {
  if (!plan || !t) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  Timing &tm = plan->p.timing;
  if (!tm.on || !tm.valid) return fail(DFDM_ERR_INVALID_ARG, "no timed apply");
  return guarded([&]() -> dfdm_status {
    std::memset(t, 0, sizeof(*t));
    for (const auto &s : tm.segs) {
      DFDM_CUDA_TRY(cudaEventSynchronize(s.b));
      float ms = 0.f;
      DFDM_CUDA_TRY(cudaEventElapsedTime(&ms, s.a, s.b));
      switch (s.phase) {
        case -1: t->total_ms += ms; break;
        case kPhS2M: t->s2m_ms += ms; break;
        case kPhM2M: t->m2m_ms += ms; break;
        case kPhSplit: t->split_ms += ms; break;
        case kPhL2L: t->l2l_ms += ms; break;
        case kPhL2T: t->l2t_ms += ms; break;
        case kPhNear: t->near_ms += ms; break;
        default:
          if (s.phase >= kPhM2L0 && s.phase < kPhM2L0 + 16) t->m2l_ms[s.phase - kPhM2L0] += ms;
      }
    }
    t->launches = tm.acc_launches;
    t->applies = tm.applies;
    tm.reset();
    return DFDM_OK;
  });
}

dfdm_status dfdm_apply_host(dfdm_plan plan, const void *x_host, void *y_host, int nrhs, void *stream) {
  if (!plan || !x_host || !y_host) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (nrhs < 1 || nrhs > plan->p.params.nrhs_max)
    return fail(DFDM_ERR_INVALID_ARG, "nrhs must be in 1..nrhs_max");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Plan &P = plan->p;
  const size_t elem = (P.params.precision == DFDM_FP64) ? 16 : 8;
  const size_t xb = (size_t)nrhs * P.ts.n * elem, yb = (size_t)nrhs * P.tt.n * elem;
  return guarded([&]() -> dfdm_status {
    DFDM_CUDA_TRY(cudaMemcpyAsync(P.x_dev_stage, x_host, xb, cudaMemcpyHostToDevice, st));
    dfdm_status s = dfdm_apply(plan, P.x_dev_stage, P.y_dev_stage, nrhs, stream);
    if (s != DFDM_OK) return s;
    DFDM_CUDA_TRY(cudaMemcpyAsync(y_host, P.y_dev_stage, yb, cudaMemcpyDeviceToHost, st));
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    return DFDM_OK;
  });
}

dfdm_status dfdm_plan_check(dfdm_plan plan, void *stream) {
  if (!plan) return fail(DFDM_ERR_INVALID_ARG, "NULL plan");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> dfdm_status {
    int h = 0;
    DFDM_CUDA_TRY(cudaMemcpyAsync(&h, plan->p.err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == 0) return DFDM_OK;
    DFDM_CUDA_TRY(cudaMemsetAsync(plan->p.err_flag, 0, sizeof(int), st));
    DFDM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == 1) return fail(DFDM_ERR_TIMEOUT, "a bounded device-side wait gave up");
    return fail(DFDM_ERR_NUMERIC, "a moment scale left the FP16 range");
  });
}

dfdm_status dfdm_plan_stats(dfdm_plan plan, dfdm_stats *st) {
  if (!plan || !st) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  *st = plan->p.stats;
  st->device_bytes = plan->p.device_bytes;
  return DFDM_OK;
}

dfdm_status dfdm_plan_export_tree(dfdm_plan plan, int which, int level, int64_t *nboxes,
                                  int64_t *keys, int64_t *begin, int64_t *end, int64_t *perm) {
  if (!plan || !nboxes) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (which != 0 && which != 1) return fail(DFDM_ERR_INVALID_ARG, "which must be 0 or 1");
  Plan &P = plan->p;
  if (level < 0 || level > P.depth) return fail(DFDM_ERR_INVALID_ARG, "level out of range");
  const Tree &t = (which == 0) ? P.tt : P.ts;
  return guarded([&]() -> dfdm_status {
    std::vector<int64_t> k, b, e;
    export_level(P, t, level, k, b, e, 0);
    if (keys) {
      if (*nboxes < (int64_t)k.size()) throw Error{DFDM_ERR_INVALID_ARG, "*nboxes too small"};
      std::memcpy(keys, k.data(), k.size() * 8);
      if (begin) std::memcpy(begin, b.data(), b.size() * 8);
      if (end) std::memcpy(end, e.data(), e.size() * 8);
    }
    *nboxes = (int64_t)k.size();
    if (perm) {
      std::vector<int32_t> hp(t.n);
      DFDM_CUDA_TRY(cudaMemcpy(hp.data(), t.perm, t.n * 4, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < t.n; ++i) perm[i] = hp[i];
    }
    return DFDM_OK;
  });
}

dfdm_status dfdm_plan_export_offsets(dfdm_plan plan, int level, int alpha_index, int32_t *count,
                                     int32_t *offsets, int32_t *dirs) {
  if (!plan || !count) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  Plan &P = plan->p;
  if (level < 0 || level > P.depth) return fail(DFDM_ERR_INVALID_ARG, "level out of range");
  if (alpha_index < 0 || alpha_index > 7) return fail(DFDM_ERR_INVALID_ARG, "alpha_index out of range");
  const LevelPlan &L = P.levels[level];
  const auto &ops = L.alpha_ops[alpha_index];
  if (offsets) {
    if (*count < (int32_t)ops.size()) return fail(DFDM_ERR_INVALID_ARG, "*count too small");
    for (size_t i = 0; i < ops.size(); ++i) {
      for (int a = 0; a < 3; ++a) offsets[3 * i + a] = L.off[3 * ops[i] + a];
      if (dirs) dirs[i] = L.op_dir[ops[i]];
    }
  }
  *count = (int32_t)ops.size();
  return DFDM_OK;
}

dfdm_status dfdm_direct_rows(const double *targets, int64_t n_t, const double *sources, int64_t n_s,
                             double kappa, const void *x, const int64_t *rows, int64_t nrows, void *y,
                             void *stream) {
  if (!targets || !sources || !x || !rows || !y) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (n_t < 1 || n_s < 1 || nrows < 1) return fail(DFDM_ERR_INVALID_ARG, "n_t, n_s and nrows must be >= 1");
  if (!(kappa > 0) || !std::isfinite(kappa)) return fail(DFDM_ERR_INVALID_ARG, "kappa must be finite and > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> dfdm_status {
    const int nchunk = direct_chunks(nrows, n_s);
    double2 *scratch = nullptr;
    DFDM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&scratch),
                                  (size_t)nchunk * nrows * sizeof(double2), st));
    try {
      direct_rows(targets, n_t, sources, n_s, kappa, static_cast<const double2 *>(x), rows, nrows,
                  static_cast<double2 *>(y), scratch, nchunk, st);
    } catch (...) {
      cudaFreeAsync(scratch, st);
      throw;
    }
    DFDM_CUDA_TRY(cudaFreeAsync(scratch, st));
    return DFDM_OK;
  });
}

dfdm_status dfdm_direct_rows_noalloc(const double *targets, int64_t n_t, const double *sources, int64_t n_s,
                                     double kappa, const void *x, const int64_t *rows, int64_t nrows, void *y,
                                     void *stream) {
  if (!targets || !sources || !x || !rows || !y) return fail(DFDM_ERR_INVALID_ARG, "NULL argument");
  if (n_t < 1 || n_s < 1 || nrows < 1) return fail(DFDM_ERR_INVALID_ARG, "n_t, n_s and nrows must be >= 1");
  if (!(kappa > 0) || !std::isfinite(kappa)) return fail(DFDM_ERR_INVALID_ARG, "kappa must be finite and > 0");
  if (nrows > kNoAllocScratchEntries)
    return fail(DFDM_ERR_INVALID_ARG, "nrows exceeds the fixed scratch of dfdm_direct_rows_noalloc (262144 rows)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return guarded([&]() -> dfdm_status {
    // as many source chunks as dfdm_direct_rows uses, capped by the scratch size
    const int nchunk =
        (int)std::max<int64_t>(1, std::min<int64_t>(direct_chunks(nrows, n_s), kNoAllocScratchEntries / nrows));
    double2 *scratch = noalloc_scratch();
    direct_rows(targets, n_t, sources, n_s, kappa, static_cast<const double2 *>(x), rows, nrows,
                static_cast<double2 *>(y), scratch, nchunk, st);
    return DFDM_OK;
  });
}

dfdm_status dfdm_plan_destroy(dfdm_plan plan) {
  if (!plan) return DFDM_OK;
  plan->p.free_all();
  delete plan;
  return DFDM_OK;
}

}  // extern "C"

namespace {
bool uniform_args_ok(double kappa, double eta2, double root_side, int depth, int l_hf) {
  return kappa > 0 && std::isfinite(kappa) && eta2 > 0 && std::isfinite(eta2) && root_side > 0 &&
         std::isfinite(root_side) && depth >= 0 && depth <= kMaxDepth && l_hf >= -2;
}
// The planner's tables of a uniform tree (host only: no trees, no device memory).
void uniform_plan(Plan &plan, double kappa, double eta2, double root_side, int depth, int l_hf) {
  plan.kappa = kappa;
  plan.params.eta2 = eta2;
  plan.root_side = root_side;
  plan.depth = depth;
  plan.l_hf = (l_hf == -2) ? default_l_hf(kappa, root_side, depth) : l_hf;
  if (plan.l_hf > depth) plan.l_hf = depth;
  build_levels(plan);
}
}  // namespace

extern "C" {

dfdm_status dfdm_uniform_offsets(double kappa, double eta2, double root_side, int depth, int l_hf, int level,
                                 int alpha_index, int32_t *count, int32_t *offsets, int32_t *dirs) {
  if (!count || !uniform_args_ok(kappa, eta2, root_side, depth, l_hf) || level < 0 || level > depth ||
      alpha_index < 0 || alpha_index > 7)
    return fail(DFDM_ERR_INVALID_ARG, "dfdm_uniform_offsets: invalid argument");
  return guarded([&]() -> dfdm_status {
    Plan plan;
    uniform_plan(plan, kappa, eta2, root_side, depth, l_hf);
    const LevelPlan &L = plan.levels[level];
    const auto &ops = L.alpha_ops[alpha_index];
    if (offsets) {
      if (*count < (int32_t)ops.size()) return fail(DFDM_ERR_INVALID_ARG, "*count too small");
      for (size_t i = 0; i < ops.size(); ++i) {
        for (int a = 0; a < 3; ++a) offsets[3 * i + a] = L.off[3 * ops[i] + a];
        if (dirs) dirs[i] = L.op_dir[ops[i]];
      }
    }
    *count = (int32_t)ops.size();
    return DFDM_OK;
  });
}

dfdm_status dfdm_uniform_counts(double kappa, double eta2, double root_side, int depth, int l_hf,
                                int64_t *n_coupling, int64_t *n_stored_coupling, int64_t *near_leaf_pairs) {
  if (!uniform_args_ok(kappa, eta2, root_side, depth, l_hf))
    return fail(DFDM_ERR_INVALID_ARG, "dfdm_uniform_counts: invalid argument");
  return guarded([&]() -> dfdm_status {
    Plan plan;
    uniform_plan(plan, kappa, eta2, root_side, depth, l_hf);
    // targets t of parity a on a grid of g boxes per axis whose source t - d
    // is on the grid too
    auto cnt = [](int64_t g, int a, int64_t d) -> int64_t {
      const int64_t lo = std::max<int64_t>(0, d), hi = std::min<int64_t>(g, g + d);
      if (hi <= lo) return 0;
      const int64_t first = lo + (((a - lo) % 2) + 2) % 2;
      return first >= hi ? 0 : (hi - 1 - first) / 2 + 1;
    };
    int64_t nc = 0;
    for (int l = 1; l <= depth; ++l) {
      const LevelPlan &L = plan.levels[l];
      for (int alpha = 0; alpha < 8; ++alpha)
        for (int op : L.alpha_ops[alpha]) {
          int64_t c = 1;
          for (int i = 0; i < 3; ++i) c *= cnt(L.grid, (alpha >> i) & 1, L.off[3 * op + i]);
          nc += c;
        }
    }
    int64_t np = 0;
    const int64_t g = (int64_t)1 << depth;
    for (size_t i = 0; i + 2 < plan.near_off.size(); i += 3) {
      int64_t c = 1;
      for (int k = 0; k < 3; ++k) c *= std::max<int64_t>(0, g - std::abs((int64_t)plan.near_off[i + k]));
      np += c;
    }
    if (n_coupling) *n_coupling = nc;
    if (n_stored_coupling) *n_stored_coupling = plan.n_ops;
    if (near_leaf_pairs) *near_leaf_pairs = np;
    return DFDM_OK;
  });
}

const char *dfdm_last_error(void) { return last_error(); }

const char *dfdm_version(void) { return "dfdm-gb300 0.1 (sm_103a)"; }

}  // extern "C"
