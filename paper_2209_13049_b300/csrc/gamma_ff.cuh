// Float-float Gamma products shared by several translation units: the
// operand split, float-float sums and the anti-diagonal sum of the Gamma'
// partials.
#pragma once

#include "common.cuh"

namespace lqmpc {

constexpr int kFfMaxSplits = 16;   // K splits of a float-float Gamma product

// v = h + l with h = fl32(v), l = fl32(v - h): about 48 significant bits.
__device__ __forceinline__ void split_ff(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// The split-K partials of the float-float products stay float-float: one
// (hi, lo) pair per entry of the partial buffer (the accumulators as the
// product left them; the FP64 products keep doubles there), summed on the
// FP32 pipe.  FP64 arithmetic issues at two lanes per clock per SM on this
// part, so a double per partial (two conversions and an add) and FP64 sums
// cost more than the float-float ones.
__device__ __forceinline__ float2* ff_parts(const Inst& I) { return reinterpret_cast<float2*>(I.gpart); }

// (ah, al) += (bh, bl): an error-free sum of the high parts (TwoSum), the low
// parts and that sum's error added in FP32, then renormalised (Fast2Sum).
// Commutative, so a butterfly leaves the same pair in every lane.
__device__ __forceinline__ void ff_acc(float& ah, float& al, float bh, float bl) {
    const float s = ah + bh;
    const float z = s - ah;
    const float t = (ah - (s - z)) + (bh - z);
    const float lo = (al + bl) + t;
    ah = s + lo;
    al = lo - (ah - s);
}

__device__ __forceinline__ void warp_sum_ff(float& h, float& l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_xor_sync(0xffffffffu, h, o), bl = __shfl_xor_sync(0xffffffffu, l, o);
        ff_acc(h, l, bh, bl);
    }
}

// One output of Gamma' w from the split partials of the float-float
// product (one warp, result in every lane):
//     out[t nu + c] = sum_split sum_{d=0}^{N-1-t} P[(N-1-d) nu + c, t + d],
// the partials stored skewed along the anti-diagonals, [split][vec][t][c][d],
// so the terms of one output are contiguous.
__device__ __forceinline__ double gamma_tmv_ff_gather(const Inst& I, int NV, int vec, int j, int splits) {
    const int lane = threadIdx.x & 31;
    const int nu = I.nu, N = I.N, n = I.n, t = j / nu, c = j % nu, nd = N - t;
    const float2* base = ff_parts(I) + (((size_t)vec * N + t) * nu + c) * N;
    const size_t stride = (size_t)NV * N * n;
    // every split's first 64 terms with independent loads (all in flight),
    // then any rest of long horizons
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
#pragma unroll
    for (int sp = 0; sp < kFfMaxSplits; ++sp) {
        if (sp < splits) {
            const float2* src = base + (size_t)sp * stride;
            if (lane < nd) { const float2 p = src[lane]; ff_acc(h0, l0, p.x, p.y); }
            if (lane + 32 < nd) { const float2 p = src[lane + 32]; ff_acc(h1, l1, p.x, p.y); }
        }
    }
    for (int sp = 0; sp < splits; ++sp)
        for (int d = lane + 64; d < nd; d += 32) {
            const float2 p = base[(size_t)sp * stride + d];
            ff_acc(h0, l0, p.x, p.y);
        }
    ff_acc(h0, l0, h1, l1);
    warp_sum_ff(h0, l0);
    return (double)h0 + (double)l0;
}

}  // namespace lqmpc
