// Two-level FP32 preconditioner of the condensed KKT matrix (Eq. 7), the
// tier between the FP32 factor and the FP64 one.
//
// Near the end of the interior-point iterations Sigma spans many decades,
// cond(M) 2^-24 approaches one and conjugate gradients preconditioned by the
// FP32 factor L1 (M ~ L1 L1', X1 ~ L1^{-1} its computed FP32 inverse) need
// tens of steps or diverge.  The operator those iterations see,
//     A2 = X1 M X1',
// is symmetric positive definite with a small condition number whenever they
// converge at all, so its FP32 Cholesky factor L2 (inverse X2) is accurate
// to ~2^-24 cond(A2), and Y = X2 X1 makes Y M Y' = X2 A2 X2' ~ I: the
// preconditioner P^{-1} = Y' Y.  Two things keep it that accurate:
//   - A2 is formed from the stored X1 and the exact M, without cancellation:
//     with E = M - L1 L1' and W = X1 L1 (I plus the inversion residual),
//         A2 = W W' + X1 E X1',
//     E and W from float-float sums of exact FP32 products (FMA), the two
//     FP32 products from operands of the size of their result;
//   - Y is applied as computed: Y = X2 X1 is formed in float-float (hi + lo
//     planes) and the preconditioner multiplies by both planes with
//     float-float sums, so no FP32 rounding of an inverse with large entries
//     enters (that rounding limits the FP32 tier's own X1 to ~2^-24 cond(L1)).
// The conjugate gradients keep their FP64-accurate products with M.
//
// Sequence (per instance, batches along grid.y), after the FP64 formation:
//     M32 = fl(M64)                   k_x2_round   (relative diagonal shift on retries)
//     L1, X1   = FP32 Cholesky + inverse of M32    (the FP32 tier's kernels)
//     S1  = E  = M64 - L1 L1'         k_x2_resid   (full symmetric)
//     S2b = W  = X1 L1                k_x2_trimul  (lower)
//     S2a = G  = X1 E                 k_x2_gemm
//     M32 = A2 = G X1' + W W'         k_x2_gemm    (lower)
//     S1  = X1                        k_x2_copy
//     L2, X2   = FP32 Cholesky + inverse of M32
//     S2a + S2b = Y = X2 X1           k_x2_trimul  (float-float, lower)
//     Xinv32 / Xlo32 = Y, XinvT32 / XloT32 = Y'    k_x2_copy
// Scratch: S1 = Xlo32 (n^2 floats; free until k_x2_copy writes Y's low plane
// there, after the last read of S1; not Tinv32, which the grid-cooperative
// Cholesky uses for its inverse), S2a / S2b = the two halves of M64 (free
// once E is formed).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

namespace {

constexpr int kXb = 32;          // tile edge (and K step) of every kernel here

__device__ __forceinline__ float* x2_s1(const Inst& I) { return I.Xlo32; }
__device__ __forceinline__ float* x2_s2a(const Inst& I) { return reinterpret_cast<float*>(I.M64); }
__device__ __forceinline__ float* x2_s2b(const Inst& I) {
    return reinterpret_cast<float*>(I.M64) + (size_t)I.n * I.n;
}

// tile index t of the lower triangle of nt x nt tiles -> (ti, tj), ti >= tj
__device__ __forceinline__ void lower_tile(int t, int& ti, int& tj) {
    int i = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    ti = i;
    tj = t - i * (i + 1) / 2;
}

}  // namespace

// M32 = fl(M64) on the lower triangle, the diagonal scaled by (1 + shift).
__global__ void k_x2_round(const Inst* __restrict__ insts, int flags, double shift) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int n = I.n;
    const size_t nn = (size_t)n * n;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        if (i < j) continue;
        double v = I.M64[e];
        if (i == j) v *= 1.0 + shift;
        I.M32[e] = (float)v;
    }
}

// S1 = E = M64 - L1 L1' (symmetric, both triangles written), L1 the lower
// triangle of M32.  One CTA per 32 x 32 lower tile, 256 threads, four
// entries each (row tid % 32, columns tid / 32 + 8 q); the products
// L1(i, k) L1(j, k) are exact as p + e (FMA) and summed in float-float.
__global__ void __launch_bounds__(256) k_x2_resid(const Inst* __restrict__ insts, int flags) {
    pdl_wait();
    __shared__ float As[kXb][kXb + 1], Bs[kXb][kXb + 1];
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    const int n = I.n, nt = (n + kXb - 1) / kXb;
    if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
    int ti, tj;
    lower_tile(blockIdx.x, ti, tj);
    const float* L = I.M32;
    const int r = threadIdx.x % kXb, cb = threadIdx.x / kXb;
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kt = 0; kt <= tj; ++kt) {   // L1(j, k) = 0 for k > j
        for (int e = threadIdx.x; e < kXb * kXb; e += blockDim.x) {
            const int rr = e % kXb, kk = e / kXb, k = kt * kXb + kk;
            const int ia = ti * kXb + rr, ib = tj * kXb + rr;
            As[rr][kk] = (ia < n && k < n && k <= ia) ? L[(size_t)ia + (size_t)n * k] : 0.f;
            Bs[rr][kk] = (ib < n && k < n && k <= ib) ? L[(size_t)ib + (size_t)n * k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kXb; ++kk) {
            const float a = As[r][kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float b = Bs[cb + 8 * q][kk];
                const float p = a * b;
                const float pe = fmaf(a, b, -p);
                const float s = sh[q] + p;
                const float z = s - sh[q];
                sl[q] += ((sh[q] - (s - z)) + (p - z)) + pe;
                sh[q] = s;
            }
        }
        __syncthreads();
    }
    float* E = x2_s1(I);
    const int i = ti * kXb + r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = tj * kXb + cb + 8 * q;
        if (i < n && j < n && j <= i) {
            const float v = (float)((I.M64[(size_t)i + (size_t)n * j] - (double)sh[q]) - (double)sl[q]);
            E[(size_t)i + (size_t)n * j] = v;
            E[(size_t)j + (size_t)n * i] = v;
        }
    }
}

// C = A B for two lower-triangular FP32 operands with float-float sums of
// the exact products (lower 32 x 32 tiles, K from tj*32 to ti*32+31):
//   mode 0: S2b = fl(W),  W = X1 L1    A = Xinv32, B = M32 (L1)
//   mode 1: S2a + S2b = Y = X2 X1     A = Xinv32 (X2), B = S1 (X1)
__global__ void __launch_bounds__(256) k_x2_trimul(const Inst* __restrict__ insts, int flags, int mode) {
    pdl_wait();
    __shared__ float As[kXb][kXb + 1], Bs[kXb][kXb + 1];
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    const int n = I.n, nt = (n + kXb - 1) / kXb;
    if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
    int ti, tj;
    lower_tile(blockIdx.x, ti, tj);
    const float* A = I.Xinv32;
    const float* B = mode == 0 ? I.M32 : x2_s1(I);
    const int r = threadIdx.x % kXb, cb = threadIdx.x / kXb;
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kt = tj; kt <= ti; ++kt) {
        for (int e = threadIdx.x; e < kXb * kXb; e += blockDim.x) {
            const int rr = e % kXb, kk = e / kXb, k = kt * kXb + kk;
            const int ia = ti * kXb + rr;          // A(ia, k), k <= ia
            As[rr][kk] = (ia < n && k < n && k <= ia) ? A[(size_t)ia + (size_t)n * k] : 0.f;
            const int jb = tj * kXb + kk, kb = kt * kXb + rr;   // B(kb, jb), kb >= jb
            Bs[rr][kk] = (jb < n && kb < n && kb >= jb) ? B[(size_t)kb + (size_t)n * jb] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kXb; ++kk) {
            const float a = As[r][kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float b = Bs[kk][cb + 8 * q];
                const float p = a * b;
                const float pe = fmaf(a, b, -p);
                const float s = sh[q] + p;
                const float z = s - sh[q];
                sl[q] += ((sh[q] - (s - z)) + (p - z)) + pe;
                sh[q] = s;
            }
        }
        __syncthreads();
    }
    const int i = ti * kXb + r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = tj * kXb + cb + 8 * q;
        if (i >= n || j >= n || j > i) continue;
        const size_t e = (size_t)i + (size_t)n * j;
        if (mode == 0) {
            x2_s2b(I)[e] = sh[q] + sl[q];
        } else {   // renormalised hi + lo
            const float hi = sh[q] + sl[q];
            x2_s2a(I)[e] = hi;
            x2_s2b(I)[e] = sl[q] - (hi - sh[q]);
        }
    }
}

// FP32 products of the two-level preconditioner, C = A B over 32 x 32 output
// tiles (column-major n x n), K limited to where the operands are nonzero:
//   mode 0: S2a = G = X1 E                 A = X1 (Xinv32, k <= i), B = E (S1); all tiles
//   mode 1: M32 = A2 = G X1' + W W'        A = G (S2a), B = X1' (XinvT32, k <= j), then
//                                          A = W (S2b, k <= i), B = W' (k <= j); lower tiles
// 256 threads, four entries each (row tid % 32, columns tid / 32 + 8 q), K in
// steps of 32 staged through shared memory with coalesced loads.
__global__ void __launch_bounds__(256) k_x2_gemm(const Inst* __restrict__ insts, int flags, int mode) {
    pdl_wait();
    __shared__ float As[kXb][kXb + 1], Bs[kXb][kXb + 1];
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    const int n = I.n, nt = (n + kXb - 1) / kXb;
    int ti, tj;
    if (mode == 0) {
        if ((int)blockIdx.x >= nt * nt) return;
        ti = blockIdx.x % nt;
        tj = blockIdx.x / nt;
    } else {
        if ((int)blockIdx.x >= nt * (nt + 1) / 2) return;
        lower_tile(blockIdx.x, ti, tj);
    }
    const int r = threadIdx.x % kXb, cb = threadIdx.x / kXb;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    // pass 0: X1 E (mode 0) or G X1' (mode 1); pass 1 (mode 1): W W'
    for (int pass = 0; pass < (mode == 0 ? 1 : 2); ++pass) {
        const float* A = mode == 0 ? I.Xinv32 : (pass == 0 ? x2_s2a(I) : x2_s2b(I));
        const int kend = min(n, ((mode == 0 ? ti : tj) + 1) * kXb);
        const bool a_lower = mode == 0 || pass == 1;   // A(i, k) = 0 for k > i
        for (int k0 = 0; k0 < kend; k0 += kXb) {
            for (int e = threadIdx.x; e < kXb * kXb; e += blockDim.x) {
                const int rr = e % kXb, kk = e / kXb, i = ti * kXb + rr, k = k0 + kk;
                As[rr][kk] = (i < n && k < kend && (!a_lower || k <= i)) ? A[(size_t)i + (size_t)n * k] : 0.f;
                if (mode == 1 && pass == 1) {   // W'(k, j) = W(j, k): j fastest
                    const int jj = e % kXb, k2 = k0 + e / kXb, j = tj * kXb + jj;
                    Bs[e / kXb][jj] = (j < n && k2 < kend && k2 <= j) ? x2_s2b(I)[(size_t)j + (size_t)n * k2] : 0.f;
                } else {                        // B(k, j) column-major: k fastest
                    const int j = tj * kXb + kk;   // here kk runs over columns, rr over k
                    const int k2 = k0 + rr;
                    float bv = 0.f;
                    if (j < n && k2 < kend) {
                        if (mode == 0) bv = x2_s1(I)[(size_t)k2 + (size_t)n * j];
                        else if (k2 <= j) bv = I.XinvT32[(size_t)k2 + (size_t)n * j];
                    }
                    Bs[rr][kk] = bv;
                }
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < kXb; ++kk) {
                const float a = As[r][kk];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(a, Bs[kk][cb + 8 * q], acc[q]);
            }
            __syncthreads();
        }
    }
    const int i = ti * kXb + r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = tj * kXb + cb + 8 * q;
        if (i >= n || j >= n) continue;
        if (mode == 0) x2_s2a(I)[(size_t)i + (size_t)n * j] = acc[q];
        else if (j <= i) I.M32[(size_t)i + (size_t)n * j] = acc[q];
    }
}

// what 0: S1 = Xinv32 (keep X1); 1: Xinv32 / Xlo32 = Y (lower), XinvT32 /
// XloT32 = Y' (upper) from S2a / S2b
__global__ void k_x2_copy(const Inst* __restrict__ insts, int flags, int what) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    const int n = I.n;
    const size_t nn = (size_t)n * n;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += stride) {
        if (what == 0) {
            x2_s1(I)[e] = I.Xinv32[e];
        } else {
            const int i = (int)(e % n), j = (int)(e / n);
            if (i < j) continue;
            const size_t t = (size_t)j + (size_t)n * i;
            const float hi = x2_s2a(I)[e], lo = x2_s2b(I)[e];
            I.Xinv32[e] = hi;
            I.Xlo32[e] = lo;
            I.XinvT32[t] = hi;
            I.XloT32[t] = lo;
        }
    }
}

void launch_x2_round(const Inst* d_insts, int count, int max_n, int flags, cudaStream_t st, double shift) {
    const int blocks = per_instance_blocks(std::min(1024, ((max_n * max_n) + 255) / 256), count);
    LQ_LAUNCH(lq_pdl(k_x2_round, dim3(blocks, count), 256, 0, st, d_insts, flags, shift));
}

void launch_x2_refine(const Inst* d_insts, int count, int max_n, int flags, cudaStream_t st) {
    const int nt = (max_n + kXb - 1) / kXb;
    const int cblocks = per_instance_blocks(std::min(1024, ((max_n * max_n) + 255) / 256), count);
    LQ_LAUNCH(lq_pdl(k_x2_resid, dim3(nt * (nt + 1) / 2, count), 256, 0, st, d_insts, flags));
    LQ_LAUNCH(lq_pdl(k_x2_trimul, dim3(nt * (nt + 1) / 2, count), 256, 0, st, d_insts, flags, 0));
    LQ_LAUNCH(lq_pdl(k_x2_gemm, dim3(nt * nt, count), 256, 0, st, d_insts, flags, 0));
    LQ_LAUNCH(lq_pdl(k_x2_gemm, dim3(nt * (nt + 1) / 2, count), 256, 0, st, d_insts, flags, 1));
    LQ_LAUNCH(lq_pdl(k_x2_copy, dim3(cblocks, count), 256, 0, st, d_insts, flags, 0));
}

void launch_x2_combine(const Inst* d_insts, int count, int max_n, int flags, cudaStream_t st) {
    const int nt = (max_n + kXb - 1) / kXb;
    const int cblocks = per_instance_blocks(std::min(1024, ((max_n * max_n) + 255) / 256), count);
    LQ_LAUNCH(lq_pdl(k_x2_trimul, dim3(nt * (nt + 1) / 2, count), 256, 0, st, d_insts, flags, 1));
    LQ_LAUNCH(lq_pdl(k_x2_copy, dim3(cblocks, count), 256, 0, st, d_insts, flags, 1));
}

}  // namespace lqmpc
