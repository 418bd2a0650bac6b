// Launcher of the Eq. 7 quantisation error (quant.cu).
#pragma once

#include "ofu_internal.cuh"

namespace ofu {

// sum over the leaves of v of |u(l) - mean of `fine` over leaf l|, into
// *err_dev (device double).  fine: device float32 [8^D] in Morton order;
// cfine: scratch of 8^D + 1 doubles; terms: scratch of n + 1 doubles; tmp:
// scan scratch of scan_tmp_items<double>(max(8^D, n)) doubles.
cudaError_t launch_quant_error(View v, const float* u, const float* fine, double* cfine,
                               double* terms, double* tmp, cudaStream_t s);

}  // namespace ofu
