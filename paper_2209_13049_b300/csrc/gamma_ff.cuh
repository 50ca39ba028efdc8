// Float-float Gamma products shared by several translation units: the
// operand split and the anti-diagonal sum of the Gamma' partials.
#pragma once

#include "common.cuh"

namespace lqmpc {

constexpr int kFfMaxSplits = 16;   // K splits of a float-float Gamma product

// v = h + l with h = fl32(v), l = fl32(v - h): about 48 significant bits.
__device__ __forceinline__ void split_ff(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// One output of Gamma' w from the split partials of the float-float
// product (one warp, result in every lane):
//     out[t nu + c] = sum_split sum_{d=0}^{N-1-t} P[(N-1-d) nu + c, t + d],
// the partials stored skewed along the anti-diagonals, [split][vec][t][c][d],
// so the terms of one output are contiguous.
__device__ __forceinline__ double gamma_tmv_ff_gather(const Inst& I, int NV, int vec, int j, int splits) {
    const int lane = threadIdx.x & 31;
    const int nu = I.nu, N = I.N, n = I.n, t = j / nu, c = j % nu, nd = N - t;
    const double* base = I.gpart + (((size_t)vec * N + t) * nu + c) * N;
    const size_t stride = (size_t)NV * N * n;
    // every split's first 64 terms with independent loads (all in flight),
    // then any rest of long horizons
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int sp = 0; sp < kFfMaxSplits; ++sp) {
        if (sp < splits) {
            const double* src = base + (size_t)sp * stride;
            if (lane < nd) s0 += src[lane];
            if (lane + 32 < nd) s1 += src[lane + 32];
        }
    }
    for (int sp = 0; sp < splits; ++sp)
        for (int d = lane + 64; d < nd; d += 32) s0 += base[(size_t)sp * stride + d];
    return warp_sum(s0 + s1);
}

}  // namespace lqmpc
