// Dense Cholesky factorisation M = L L' and the two triangular solves of the
// condensed system (Eq. 7: M is positive definite, factor and solve).
//
// Right-looking blocked algorithm with 32-wide panels.  For panel k one
// launch factors the diagonal block (one warp per CTA, each CTA redundantly)
// and solves the panel rows below it (one row per lane); a second launch
// applies the rank-32 update to the trailing lower triangle in 32 x 32 tiles.
// A non-positive (or NaN) pivot records its global index + 1 in Scal::info and
// every later step of the iteration is skipped.
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

constexpr int kNb = 32;

template <typename T>
__device__ __forceinline__ T* kkt_mat(const Inst& I) {
    return sizeof(T) == 8 ? (T*)I.M64 : (T*)I.M32;
}

template <typename T> __device__ __forceinline__ T sqrt_t(T v);
template <> __device__ __forceinline__ double sqrt_t<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float sqrt_t<float>(float v) { return sqrtf(v); }

template <typename T>
__global__ void __launch_bounds__(32) k_potrf_panel(const Inst* __restrict__ insts, int k, int force) {
    const Inst& I = insts[blockIdx.y];
    if (!force && I.sc->done) return;
    if (I.sc->info) return;
    const int n = I.n;
    const int nt = (n + kNb - 1) / kNb;
    if (k >= nt) return;
    const int p = k + blockIdx.x;
    if (p >= nt) return;
    T* M = kkt_mat<T>(I);
    const int lane = threadIdx.x;
    const int k0 = k * kNb, kn = min(kNb, n - k0);
    __shared__ T Ld[kNb][kNb + 1];
    __shared__ T X[kNb][kNb + 1];
    for (int c = 0; c < kNb; ++c) {
        T v = (c == lane) ? T(1) : T(0);
        if (lane < kn && c < kn && c <= lane) v = M[(size_t)(k0 + lane) + (size_t)n * (k0 + c)];
        Ld[lane][c] = v;
    }
    __syncwarp();
    for (int j = 0; j < kNb; ++j) {
        T djj = Ld[j][j];
        if (!(djj > T(0))) {          // uniform across the warp
            if (lane == 0 && blockIdx.x == 0) atomicCAS(&I.sc->info, 0, k0 + j + 1);
            return;
        }
        T d = sqrt_t<T>(djj);
        __syncwarp();
        if (lane == j) Ld[j][j] = d;
        if (lane > j) Ld[lane][j] = Ld[lane][j] / d;
        __syncwarp();
        if (lane > j) {
            T lij = Ld[lane][j];
            for (int l = j + 1; l <= lane; ++l) Ld[lane][l] -= lij * Ld[l][j];
        }
        __syncwarp();
    }
    if (blockIdx.x == 0) {
        if (lane < kn)
            for (int c = 0; c <= lane; ++c) M[(size_t)(k0 + lane) + (size_t)n * (k0 + c)] = Ld[lane][c];
        return;
    }
    // row tile p: X = A_pk L_kk^{-T}
    const int row = p * kNb + lane;
    for (int c = 0; c < kNb; ++c)
        X[lane][c] = (row < n && c < kn) ? M[(size_t)row + (size_t)n * (k0 + c)] : T(0);
    __syncwarp();
    if (row < n) {
        for (int c = 0; c < kn; ++c) {
            T v = X[lane][c];
            for (int m = 0; m < c; ++m) v -= X[lane][m] * Ld[c][m];
            X[lane][c] = v / Ld[c][c];
        }
    }
    __syncwarp();
    if (row < n)
        for (int c = 0; c < kn; ++c) M[(size_t)row + (size_t)n * (k0 + c)] = X[lane][c];
}

// A_pq -= L_pk L_qk' for trailing tiles k < q <= p.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_update(const Inst* __restrict__ insts, int k, int force) {
    const Inst& I = insts[blockIdx.y];
    if (!force && I.sc->done) return;
    if (I.sc->info) return;
    const int n = I.n;
    const int nt = (n + kNb - 1) / kNb;
    const int m = nt - k - 1;                 // trailing tiles per side
    if (m <= 0) return;
    const int t = blockIdx.x;
    if (t >= m * (m + 1) / 2) return;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    const int b = t - a * (a + 1) / 2;
    const int p = k + 1 + a, q = k + 1 + b;
    T* M = kkt_mat<T>(I);
    const int k0 = k * kNb, kn = min(kNb, n - k0);
    __shared__ T Lp[kNb][kNb + 1];
    __shared__ T Lq[kNb][kNb + 1];
    for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
        int r = e % kNb, c = e / kNb;
        int rp = p * kNb + r, rq = q * kNb + r;
        Lp[r][c] = (rp < n && c < kn) ? M[(size_t)rp + (size_t)n * (k0 + c)] : T(0);
        Lq[r][c] = (rq < n && c < kn) ? M[(size_t)rq + (size_t)n * (k0 + c)] : T(0);
    }
    __syncthreads();
    const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
    T acc[4] = {0, 0, 0, 0};
#pragma unroll 8
    for (int c = 0; c < kNb; ++c) {
        T lp = Lp[ty][c];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] += lp * Lq[tx * 4 + e][c];
    }
    const int row = p * kNb + ty;
    if (row < n) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int col = q * kNb + tx * 4 + e;
            if (col < n && col <= row) M[(size_t)row + (size_t)n * col] -= acc[e];
        }
    }
}

// Solve L L' x = b for one right-hand side per instance (one CTA each).  The
// FP32 variant scales b by 1/||b||_inf so the working values stay O(1).
template <typename T>
__global__ void __launch_bounds__(1024) k_chol_solve(const Inst* __restrict__ insts, int in_role,
                                                     int out_role, int flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* y = (T*)smem_raw;
    __shared__ double red[32];
    __shared__ double s_scale;
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    if (I.sc->info) return;
    const int n = I.n;
    const T* L = kkt_mat<T>(I);
    const double* bin = role_ptr(I, in_role);
    double* xout = role_ptr(I, out_role);
    double bm = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) bm = fmax(bm, fabs(bin[j]));
    bm = block_reduce<1>(bm, red);
    if (threadIdx.x == 0) s_scale = (sizeof(T) == 4 && bm > 0.0) ? bm : 1.0;
    __syncthreads();
    const double sc = s_scale;
    for (int j = threadIdx.x; j < n; j += blockDim.x) y[j] = (T)(bin[j] / sc);
    __syncthreads();
    const int nt = (n + kNb - 1) / kNb;
    const unsigned full = 0xffffffffu;
    for (int kb = 0; kb < nt; ++kb) {
        const int k0 = kb * kNb, kn = min(kNb, n - k0);
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            T v = lane < kn ? y[k0 + lane] : T(0);
            for (int j = 0; j < kn; ++j) {
                T yj = __shfl_sync(full, v, j) / L[(size_t)(k0 + j) * (n + 1)];
                if (lane == j) v = yj;
                if (lane > j && lane < kn) v -= L[(size_t)(k0 + lane) + (size_t)n * (k0 + j)] * yj;
            }
            if (lane < kn) y[k0 + lane] = v;
        }
        __syncthreads();
        for (int i = k0 + kn + threadIdx.x; i < n; i += blockDim.x) {
            T acc = 0;
            for (int j = 0; j < kn; ++j) acc += L[(size_t)i + (size_t)n * (k0 + j)] * y[k0 + j];
            y[i] -= acc;
        }
        __syncthreads();
    }
    for (int kb = nt - 1; kb >= 0; --kb) {
        const int k0 = kb * kNb, kn = min(kNb, n - k0);
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            T v = lane < kn ? y[k0 + lane] : T(0);
            for (int j = kn - 1; j >= 0; --j) {
                T xj = __shfl_sync(full, v, j) / L[(size_t)(k0 + j) * (n + 1)];
                if (lane == j) v = xj;
                if (lane < j) v -= L[(size_t)(k0 + j) + (size_t)n * (k0 + lane)] * xj;
            }
            if (lane < kn) y[k0 + lane] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k0; i += blockDim.x) {
            T acc = 0;
            const T* Li = L + (size_t)n * i;
            for (int j = 0; j < kn; ++j) acc += Li[k0 + j] * y[k0 + j];
            y[i] -= acc;
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) xout[j] = (double)y[j] * sc;
}

// ---------------------------------------------------------------------------

void launch_potrf(const Inst* d_insts, int count, int max_n, int fp64, int force, cudaStream_t st) {
    const int nt = (max_n + kNb - 1) / kNb;
    for (int k = 0; k < nt; ++k) {
        dim3 g1(nt - k, count);
        int m = nt - k - 1;
        dim3 g2(m * (m + 1) / 2 > 0 ? m * (m + 1) / 2 : 1, count);
        if (fp64) {
            LQ_LAUNCH(k_potrf_panel<double><<<g1, 32, 0, st>>>(d_insts, k, force));
            if (m > 0) LQ_LAUNCH(k_potrf_update<double><<<g2, 256, 0, st>>>(d_insts, k, force));
        } else {
            LQ_LAUNCH(k_potrf_panel<float><<<g1, 32, 0, st>>>(d_insts, k, force));
            if (m > 0) LQ_LAUNCH(k_potrf_update<float><<<g2, 256, 0, st>>>(d_insts, k, force));
        }
    }
}

void launch_chol_solve(const Inst* d_insts, int count, int max_n, int fp64, int in_role,
                       int out_role, int flags, cudaStream_t st) {
    size_t smem = (size_t)max_n * (fp64 ? 8 : 4);
    if (fp64) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_chol_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(k_chol_solve<double><<<dim3(1, count), 1024, smem, st>>>(d_insts, in_role, out_role, flags));
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_chol_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(k_chol_solve<float><<<dim3(1, count), 1024, smem, st>>>(d_insts, in_role, out_role, flags));
    }
}

}  // namespace lqmpc
