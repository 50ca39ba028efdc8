// Reciprocal square root for the FP32 diagonal factorisations: rsqrtf
// refined by one Newton step (about one ulp; the factor is a
// preconditioner), so a factorisation's serial chain has no division.
#pragma once

#include <cuda_runtime.h>

namespace lqmpc {

__device__ __forceinline__ float rsqrt_refined(float d) {
    float r = rsqrtf(d);
    return r * (1.5f - 0.5f * d * r * r);
}

}  // namespace lqmpc
