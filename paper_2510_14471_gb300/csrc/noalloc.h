// Allocation-free per-block least squares (see glm_sur_ols_static).
#pragma once
#include <cuda_runtime.h>

#include "glm_sur.h"
#include "internal.h"

namespace glmsur {

// Size of the library's fixed device scratch array (doubles): 4 MiB.
constexpr long long kOlsScratchDoubles = 1LL << 19;

glm_sur_status ols_static(const Geom& gm, const double* Q64, const double* R, const double* Y, int64_t ldy, int k,
                          double* b, int64_t ldb, int sms, cudaStream_t s);

}  // namespace glmsur
