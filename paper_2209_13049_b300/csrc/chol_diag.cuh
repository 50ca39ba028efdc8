// Pivots of the diagonal-block factorisations.
//
// rsqrt_refined (FP32 dataflow factor): rsqrtf refined by one Newton step
// (about one ulp; the factor is a preconditioner), so the serial chain has no
// division.
//
// pivot_t: d = sqrt(v) and 1/d.  FP32 takes sqrtf and a division.  FP64
// starts from the FP32 reciprocal square root and takes two Newton steps
// r <- r + r (1 - v r^2) / 2 (quadratic convergence: 2^-22, 2^-43, then
// rounding), so the pivot chain holds no FP64 square root or division: on
// this part those take about 650 and 430 cycles of latency against 64 for an
// FP64 FMA.
#pragma once

#include <cuda_runtime.h>

namespace lqmpc {

__device__ __forceinline__ float rsqrt_refined(float d) {
    float r = rsqrtf(d);
    return r * (1.5f - 0.5f * d * r * r);
}

template <typename T> __device__ __forceinline__ void pivot_t(T v, T& d, T& rd);
template <> __device__ __forceinline__ void pivot_t<float>(float v, float& d, float& rd) {
    d = sqrtf(v);
    rd = 1.0f / d;
}
template <> __device__ __forceinline__ void pivot_t<double>(double v, double& d, double& rd) {
    if (v > 1e-30 && v < 1e30) {   // the FP32 seed is in range
        double r = (double)rsqrtf((float)v);
        double e = fma(-v * r, r, 1.0);
        r = fma(0.5 * r, e, r);
        e = fma(-v * r, r, 1.0);
        r = fma(0.5 * r, e, r);
        rd = r;
        d = v * r;
    } else {
        d = sqrt(v);
        rd = 1.0 / d;
    }
}

template <typename T> __device__ __forceinline__ T fma_t(T a, T b, T c);
template <> __device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> __device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }

}  // namespace lqmpc
