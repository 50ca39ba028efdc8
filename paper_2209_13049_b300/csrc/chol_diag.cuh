// Cholesky factor of one 32 x 32 diagonal block in the registers of one
// warp (lane i holds row i), shared by the blocked factorisations.
//
// Right-looking factorisation: at step q the pivot d_q = a_qq is broadcast,
// column q is scaled by 1/sqrt(d_q) and the trailing rows are updated by
// shuffles.  The FP32 version takes 1/sqrt(d) from rsqrtf refined by one
// Newton step (about one ulp: the factor is a preconditioner), and hands the
// reciprocal of each lane's own pivot back for the inverse, so the serial
// chain has no division.
#pragma once

#include <cuda_runtime.h>

namespace lqmpc {

__device__ __forceinline__ float rsqrt_refined(float d) {
    float r = rsqrtf(d);
    return r * (1.5f - 0.5f * d * r * r);
}

// a: row `lane` of the block (entries c > lane ignored).  On return a holds
// row `lane` of L (zeros above the diagonal) and rdiag = 1 / l_{lane,lane}.
// Returns 0, or q + 1 for the first non-positive pivot q (a then undefined).
__device__ __forceinline__ int diag_factor(float (&a)[32], float& rdiag) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int fail = 0;
    rdiag = 1.f;
#pragma unroll
    for (int c = 0; c < 32; ++c) if (c > lane) a[c] = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const float dqq = __shfl_sync(full, a[q], q);
        if (!(dqq > 0.f) && !fail) fail = q + 1;
        const float r = rsqrt_refined(fail ? 1.f : dqq);
        if (lane == q) rdiag = r;
        const float liq = lane > q ? a[q] * r : (lane == q ? dqq * r : 0.f);
        a[q] = liq;
#pragma unroll
        for (int c = q + 1; c < 32; ++c) {
            const float lcq = __shfl_sync(full, liq, c);
            if (lane >= c) a[c] = fmaf(-liq, lcq, a[c]);
        }
    }
    return fail;
}

}  // namespace lqmpc
