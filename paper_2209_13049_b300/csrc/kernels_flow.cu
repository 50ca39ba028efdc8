// Dataflow Cholesky factorisation with the inverse of the factor (the FP32
// preconditioner of the mixed-precision solves, Eq. 7's M = L L') for one
// instance of n <= 544, one CTA per 32-wide block column.
//
// CTA j keeps its block column (rows 32j..n-1) in shared memory and is
// left-looking: it subtracts L_{:,k} L_{j,k}' for every earlier block column
// k as soon as CTA k has published it, factors its diagonal block in
// registers, solves the rows below by the inverse of that block, and
// publishes the column.  Then it forms block column j of X = L^{-1} by
// forward substitution down the column, X_pj = -L_pp^{-1} sum_{k=j}^{p-1}
// L_pk X_kj, consuming block columns p > j as they appear (L_pp^{-1} is
// published in X's diagonal block).  No grid-wide barrier: the critical path
// is one diagonal factorisation per block column plus its last update.
//
// Publication: a block column is written with L2-coherent stores, fenced,
// then its flag is set to the launch's epoch; readers poll the flag (bounded:
// a wait that gives up raises Scal::err bit 4 and the kernel still runs to
// its end) and read with L1-bypassing loads.  The epoch advances when the
// last CTA finishes, so flags never need clearing.  A non-positive pivot is
// recorded in Scal::info; every CTA still publishes, so nobody waits forever.
#include "chol_diag.cuh"
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

namespace {

constexpr int kFb = 32;
constexpr int kFlowMaxN = 544;          // three [32 x rows] FP32 panels fit shared memory
constexpr uint32_t kFlowSpin = 1u << 22;

__device__ __forceinline__ int ld_flag(const int* p) { return *(const volatile int*)p; }

// 16-byte global -> shared copy through L2 only (other CTAs' data is read
// after their flag), zero-filled past `bytes` (0..16).
__device__ __forceinline__ void cpa16(float* dst, const float* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Rows [row0, row0 + rows) of `cols` consecutive columns starting at column
// col0 of the column-major n x n matrix M into dst[c * ld + r] (zeros for
// r in [rows, ld)).  Vector copies when every column start is 16-byte
// aligned (n and row0 multiples of 4), scalar L2 loads otherwise.
__device__ void stage_cols(float* dst, int ld, const float* M, int n, int row0, int rows, int col0, int cols,
                           bool vec) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (vec) {
        const int q4 = ld / 4;
        for (int e = threadIdx.x; e < cols * q4; e += blockDim.x) {
            const int c = e / q4, r = 4 * (e % q4);
            const int left = rows - r;
            const int bytes = left >= 4 ? 16 : (left > 0 ? 4 * left : 0);
            const float* src = M + (size_t)n * (col0 + c) + row0 + (left > 0 ? r : 0);
            cpa16(dst + (size_t)c * ld + r, src, bytes);
        }
        cpa_wait_all();
    } else {
        for (int c = warp; c < cols; c += nw)
            for (int r = lane; r < ld; r += 32) dst[(size_t)c * ld + r] = r < rows ? __ldcg(M + (size_t)n * (col0 + c) + row0 + r) : 0.f;
    }
}

// Thread 0 waits for flag == ep (bounded), then the block proceeds.
__device__ void flow_wait(const int* flag, int ep, int* err) {
    if (threadIdx.x == 0) {
        uint32_t it = 0;
        // after one wait has given up anywhere, later waits do not spin
        while (ld_flag(flag) != ep && !(ld_flag(err) & 4)) {
            if (++it > kFlowSpin) { atomicOr(err, 4); break; }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(256, 1) k_potrf_flow(const Inst* __restrict__ insts, int flags) {
    const Inst& I = insts[0];
    if (skip_instance(I, flags)) return;           // the same decision in every CTA
    extern __shared__ __align__(16) float fsm[];
    __shared__ float D[kFb][kFb + 1], Dv[kFb][kFb + 1], Tt[kFb][kFb + 1];
    __shared__ int ep_sh;
    const int n = I.n, nt = (n + kFb - 1) / kFb, j = blockIdx.x;
    int* epoch = I.pflags;        // [0] epoch, [1] finished CTAs, [2 + k] flag of block column k
    int* done = I.pflags + 1;
    int* flg = I.pflags + 2;
    int* err = &I.sc->err;
    float* M = I.M32;
    if (threadIdx.x == 0) ep_sh = ld_flag(epoch) + 1;
    __syncthreads();
    const int ep = ep_sh;
    if (j >= nt) return;
    const int r0 = kFb * j, R = n - r0, Rp = (R + kFb - 1) / kFb * kFb;
    const int kn = min(kFb, R);                    // columns of this block column
    float* Ps = fsm;                               // [32 cols][Rp rows]
    float* Ls = Ps + (size_t)kFb * Rp;             // staging
    float* Xs = Ls + (size_t)kFb * Rp;             // block column j of X
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // own block column, padded with the identity beyond n
    const bool vec = (n % 4) == 0;
    stage_cols(Ps, Rp, M, n, r0, R, r0, kn, vec);
    for (int c = kn + warp; c < kFb; c += 8)          // identity columns of a ragged last block column
        for (int r = lane; r < Rp; r += 32) Ps[c * Rp + r] = r == c ? 1.f : 0.f;
    __syncthreads();

    // left-looking updates: A_{:,j} -= L_{:,k} L_{j,k}'  (rows r0.. of block column k)
    for (int k = 0; k < j; ++k) {
        flow_wait(flg + k, ep, err);
        stage_cols(Ls, Rp, M, n, r0, R, kFb * k, kFb, vec);
        __syncthreads();
        // Ps[c][r] -= sum_m Ls[m][r] Ls[m][c]; lane -> row, warp -> 4 columns
        for (int rb = 0; rb < Rp; rb += kFb) {
            const int r = rb + lane;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
            for (int m = 0; m < kFb; ++m) {
                const float a = Ls[m * Rp + r];
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[t] = fmaf(a, Ls[m * Rp + warp + 8 * t], acc[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) Ps[(warp + 8 * t) * Rp + r] -= acc[t];
        }
        __syncthreads();
    }

    // diagonal block: factor and invert in registers (warp 0, row i in lane i)
    if (warp == 0) {
        float a[kFb], x[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) a[c] = Ps[c * Rp + lane];
        const int fail = diag_factor_inverse(a, x);
#pragma unroll
        for (int c = 0; c < kFb; ++c) {
            D[lane][c] = c <= lane ? a[c] : 0.f;
            Dv[lane][c] = c <= lane ? x[c] : 0.f;
        }
        if (lane == 0 && fail) atomicCAS(&I.sc->info, 0, r0 + fail);
    }
    __syncthreads();

    // rows below the diagonal block: L_pj = A_pj D^{-T}, into Ls (free now);
    // the diagonal block L_jj goes to Ls as well, so Ls holds the column
    for (int rb = kFb; rb < Rp; rb += kFb) {
        const int r = rb + lane;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int m = 0; m < kFb; ++m) {
            const float a = Ps[m * Rp + r];
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[t] = fmaf(a, Dv[warp + 8 * t][m], acc[t]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) Ls[(warp + 8 * t) * Rp + r] = acc[t];
    }
    for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
        const int c = e / kFb, r = e % kFb;
        Ls[c * Rp + r] = D[r][c];
        Xs[c * Rp + r] = Dv[r][c];
    }
    __syncthreads();

    // publish block column j of L and L_jj^{-1} (X's diagonal block)
    for (int c = warp; c < kn; c += 8) {
        float* dst = M + (size_t)n * (r0 + c) + r0;
#pragma unroll 4
        for (int r = lane; r < R; r += 32)
            if (r >= c) __stcg(dst + r, Ls[c * Rp + r]);
        if (lane < kn && lane >= c) {
            const float xv = Xs[c * Rp + lane];
            __stcg(I.Xinv32 + (size_t)(r0 + lane) + (size_t)n * (r0 + c), xv);
            __stcg(I.XinvT32 + (size_t)(r0 + c) + (size_t)n * (r0 + lane), xv);
        }
    }
    __threadfence();   // every writer's stores before the flag
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(flg + j, ep);
    }

    // block column j of X: X_pj = -L_pp^{-1} sum_{k=j}^{p-1} L_pk X_kj
    for (int p = j + 1; p < nt; ++p) {
        flow_wait(flg + p, ep, err);
        const int p0 = kFb * p, pr = min(kFb, n - p0);
        const int K = p0 - r0;                       // columns r0 .. p0-1 of row block p
        // Ls[q * 32 + i] = L[p0 + i, r0 + q]
        {
            const bool v2 = vec && pr == kFb;
            if (v2) {
                for (int e = threadIdx.x; e < K * (kFb / 4); e += blockDim.x) {
                    const int q = e / (kFb / 4), i = 4 * (e % (kFb / 4));
                    cpa16(Ls + q * kFb + i, M + (size_t)(p0 + i) + (size_t)n * (r0 + q), 16);
                }
                cpa_wait_all();
            } else {
                for (int q = warp; q < K; q += 8)
                    Ls[q * kFb + lane] = lane < pr ? __ldcg(M + (size_t)(p0 + lane) + (size_t)n * (r0 + q)) : 0.f;
            }
        }
        for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
            const int r = e / kFb, c = e % kFb;   // L_pp^{-1}[r][c]
            D[r][c] = (r < pr && c < pr && c <= r) ? __ldcg(I.Xinv32 + (size_t)(p0 + r) + (size_t)n * (p0 + c)) : 0.f;
        }
        __syncthreads();
        {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < K; ++q) {
                const float a = Ls[q * kFb + lane];
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[t] = fmaf(a, Xs[(warp + 8 * t) * Rp + q], acc[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) Tt[lane][warp + 8 * t] = acc[t];
        }
        __syncthreads();
        {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
            for (int m = 0; m < kFb; ++m) {
                const float dv = D[lane][m];
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[t] = fmaf(dv, Tt[m][warp + 8 * t], acc[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) Xs[(warp + 8 * t) * Rp + (p0 - r0) + lane] = -acc[t];
        }
        __syncthreads();
    }
    // X below the diagonal block of column j (the diagonal block is already out)
    for (int c = warp; c < kn; c += 8)
        for (int r = kFb + lane; r < R; r += 32) {
            const float xv = Xs[c * Rp + r];
            I.Xinv32[(size_t)(r0 + r) + (size_t)n * (r0 + c)] = xv;
            I.XinvT32[(size_t)(r0 + c) + (size_t)n * (r0 + r)] = xv;
        }
    // the last CTA to finish advances the epoch (every CTA has read it by then)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(done, 1) == nt - 1) {
            atomicExch(done, 0);
            __threadfence();
            atomicAdd(epoch, 1);
        }
    }
}

bool potrf_flow_fits(int count, int max_n) { return count == 1 && max_n >= 1 && max_n <= kFlowMaxN; }

bool launch_potrf_flow(const Inst* d_insts, int max_n, int flags, cudaStream_t st) {
    const int nt = (max_n + kFb - 1) / kFb;
    const int Rp = nt * kFb;
    const size_t smem = 3 * sizeof(float) * kFb * (size_t)Rp;
    cudaFuncSetAttribute(k_potrf_flow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    void* args[] = {(void*)&d_insts, (void*)&flags};
    cudaEvent_t pe = prof_start(st);
    // cooperative: every block column CTA is resident, so the flag waits can end
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_potrf_flow, dim3(nt), dim3(256), args, smem, st);
    note_launches(1);
    prof_stop(st, pe, "k_potrf_flow");
    check_launch(st, "k_potrf_flow", __FILE__, __LINE__);
    return e == cudaSuccess;
}

}  // namespace lqmpc
