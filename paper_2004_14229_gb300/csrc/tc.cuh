// Tensor-core form (DFDM_TC_FP16X3): declarations.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "dfdm_internal.cuh"

namespace dfdm {

// Allocates and fills the tensor-core form's tables (split FP16 coupling
// operators, FP32 moment/local grids) after the planner ran.
void build_tc(Plan &plan, cudaStream_t st);

// Frees the host-side state of the tensor-core form (device buffers belong
// to the plan's allocation list).
void destroy_tc(Plan &plan);

// g = A v with complex64 x / y (caller order), nrhs right-hand sides.
void apply_tc(Plan &plan, const float2 *x, float2 *y, int nrhs, cudaStream_t st);

// Launch shapes of the tensor-core form that a measured tuner may set; 0 (or
// a level past the vector's end) keeps the built-in rule.
struct TcTuning {
  std::vector<int> m2l_nsplit;   // per level: CTA pairs per (tile, alpha) along the operator list
  int p2p_threads = 0;           // k_p2p_f32 block size (32, 64 or 128)
  int p2p_chunks = 0;            // target chunks per leaf
};

// Candidate M2L chunk counts of level l, the rule's first (empty: no M2L).
std::vector<int> tc_nsplit_candidates(const Plan &plan, int l);
// Candidate (threads, chunks) of k_p2p_f32, the rule's first (empty: not used).
std::vector<std::pair<int, int>> tc_p2p_candidates(const Plan &plan);
TcTuning &tc_tuning(Plan &plan);
// Times candidate shapes on whole products of x and keeps the fastest
// (dfdm_plan_autotune; cache_path may be NULL, out may be NULL).
void autotune_tc(Plan &plan, const float2 *x, const char *cache_path, cudaStream_t st, dfdm_tuning *out);
// What the launch shapes depend on: device, order, depth, per level grid,
// direction slots and operator list length, leaf count and sizes.
std::string tc_shape_key(const Plan &plan);

}  // namespace dfdm
