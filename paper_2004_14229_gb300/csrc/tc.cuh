// Tensor-core form (DFDM_TC_FP16X3): declarations.
#pragma once

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

}  // namespace dfdm
