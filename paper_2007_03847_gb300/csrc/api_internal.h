// Entry points shared between the library's own translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/fastmc.h"

namespace fmc {

// fmc_simulate with a choice of how the fused kernel combines its per-time sums:
// per_tile_partials = true writes FP32 partials per 128-sample tile and adds them
// in a fixed order (deterministic); false adds them with FP64 atomics (no
// partial buffer; the order of the FP64 additions is not fixed).
int simulate_moments(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, double* mean_dev, double* var_dev,
                     bool per_tile_partials, cudaStream_t st);

}  // namespace fmc
