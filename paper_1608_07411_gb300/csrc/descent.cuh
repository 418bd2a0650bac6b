// Launcher of the eps-L1 gradient-descent iteration (descent.cu).
#pragma once

#include "ofu_internal.cuh"

namespace ofu {

// One gradient-descent iteration with step xi on the current structure:
// q <- g / sqrt(|g|^2 + eps^2) (g = K u, q [3][stride] scratch), then
// u <- u - xi [c sum_k (u - f_k) / sqrt((u - f_k)^2 + eps^2) - lambda div q],
// ubar <- u.  Two launches on `s`.
cudaError_t launch_descent_step(View v, float* u, float* ubar, float* q, const uint32_t* soff,
                                const void* samp, bool fp16, float eps, float xi, float lambda,
                                float gamma, LeafSets dual_sets, LeafSets primal_sets,
                                cudaStream_t s);

}  // namespace ofu
