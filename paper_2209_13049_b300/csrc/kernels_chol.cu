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

// Grid-wide barrier for the cooperative factorisation kernel (all CTAs are
// co-resident by the cooperative launch).  The spin is bounded: a barrier
// that gives up raises Scal::err bit 2 and lets the kernel return.
constexpr unsigned kBarLimit = 1u << 24;

__device__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (*gen == g) {
                if (++it > kBarLimit) { ok = 0; atomicOr(err, 2); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Factor the diagonal block of panel k (warp 0, registers + shuffles) into
// Ld; returns false (uniformly) on a non-positive pivot, recorded by the CTA
// that owns the diagonal tile.
template <typename T>
__device__ bool factor_diag(const Inst& I, T* M, int k, bool owner, T (*Ld)[kNb + 1], int* fail_sh) {
    const int n = I.n, k0 = k * kNb, kn = min(kNb, n - k0);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned full = 0xffffffffu;
        T a[kNb];
#pragma unroll
        for (int c = 0; c < kNb; ++c) {
            T v = (c == lane) ? T(1) : T(0);
            if (lane < kn && c < kn && c <= lane) v = M[(size_t)(k0 + lane) + (size_t)n * (k0 + c)];
            a[c] = v;
        }
        int fail = 0;
#pragma unroll
        for (int j = 0; j < kNb; ++j) {
            if (!fail) {
                T djj = __shfl_sync(full, a[j], j);
                if (!(djj > T(0))) {
                    fail = k0 + j + 1;
                } else {
                    T d = sqrt_t<T>(djj);
                    T rd = T(1) / d;
                    T lij = lane > j ? a[j] * rd : (lane == j ? d : T(0));
                    a[j] = lij;
#pragma unroll
                    for (int c = j + 1; c < kNb; ++c) {
                        T lcj = __shfl_sync(full, lij, c);
                        if (lane >= c) a[c] -= lij * lcj;
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kNb; ++c) Ld[lane][c] = a[c];
        if (lane == 0) {
            *fail_sh = fail;
            if (fail && owner) atomicCAS(&I.sc->info, 0, fail);
        }
    }
    __syncthreads();
    return *fail_sh == 0;
}

// Panel k, row tile p (p == k: write the diagonal factor; p > k: solve the
// tile rows against it).
template <typename T>
__device__ void panel_tile(const Inst& I, int k, int p, T (*Ld)[kNb + 1], int* fail_sh) {
    T* M = kkt_mat<T>(I);
    const int n = I.n, k0 = k * kNb, kn = min(kNb, n - k0);
    if (!factor_diag<T>(I, M, k, p == k, Ld, fail_sh)) return;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (p == k) {
            if (lane < kn)
                for (int c = 0; c <= lane; ++c) M[(size_t)(k0 + lane) + (size_t)n * (k0 + c)] = Ld[lane][c];
        } else {
            const int row = p * kNb + lane;
            if (row < n) {
                T x[kNb];
#pragma unroll
                for (int c = 0; c < kNb; ++c) x[c] = c < kn ? M[(size_t)row + (size_t)n * (k0 + c)] : T(0);
#pragma unroll
                for (int c = 0; c < kNb; ++c) {
                    if (c < kn) {
                        T v = x[c];
#pragma unroll
                        for (int m = 0; m < c; ++m) v -= x[m] * Ld[c][m];
                        x[c] = v / Ld[c][c];
                    }
                }
#pragma unroll
                for (int c = 0; c < kNb; ++c)
                    if (c < kn) M[(size_t)row + (size_t)n * (k0 + c)] = x[c];
            }
        }
    }
    __syncthreads();
}

// A_pq -= L_pk L_qk' for the trailing tile (p, q), k < q <= p.
template <typename T>
__device__ void update_tile(const Inst& I, int k, int p, int q, T (*Lp)[kNb + 1], T (*Lq)[kNb + 1]) {
    T* M = kkt_mat<T>(I);
    const int n = I.n, k0 = k * kNb, kn = min(kNb, n - k0);
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
    __syncthreads();
}

// Right-looking blocked Cholesky of every participating instance in one
// cooperative launch: per panel, a panel phase (diagonal factor + panel
// solve, one row tile per work item) and an update phase (one trailing tile
// per work item), separated by grid barriers.  Instances are chosen once at
// entry (not done, no earlier failure); a pivot failure only stops that
// instance's own work.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_coop(const Inst* __restrict__ insts, int count, int max_nt,
                                                    int flags) {
    __shared__ T S1[kNb][kNb + 1];
    __shared__ T S2[kNb][kNb + 1];
    __shared__ int fail_sh;
    unsigned* bar = insts[0].bar;
    int* err = &insts[0].sc->err;
    for (int k = 0; k < max_nt; ++k) {
        // panel phase
        int total = 0;
        for (int q = 0; q < count; ++q) {
            const Inst& I = insts[q];
            const int nt = (I.n + kNb - 1) / kNb;
            if (!skip_instance(I, flags) && k < nt) total += nt - k;
        }
        for (int item = blockIdx.x; item < total; item += gridDim.x) {
            int q = 0, rem = item;
            for (;; ++q) {
                const Inst& I = insts[q];
                const int nt = (I.n + kNb - 1) / kNb;
                const int c = (!skip_instance(I, flags) && k < nt) ? nt - k : 0;
                if (rem < c) break;
                rem -= c;
            }
            const Inst& I = insts[q];
            if (!I.sc->info) panel_tile<T>(I, k, k + rem, S1, &fail_sh);
        }
        if (!grid_barrier(bar, err)) return;
        // update phase
        total = 0;
        for (int q = 0; q < count; ++q) {
            const Inst& I = insts[q];
            const int m = (I.n + kNb - 1) / kNb - k - 1;
            if (!skip_instance(I, flags) && m > 0) total += m * (m + 1) / 2;
        }
        for (int item = blockIdx.x; item < total; item += gridDim.x) {
            int q = 0, rem = item;
            for (;; ++q) {
                const Inst& I = insts[q];
                const int m = (I.n + kNb - 1) / kNb - k - 1;
                const int c = (!skip_instance(I, flags) && m > 0) ? m * (m + 1) / 2 : 0;
                if (rem < c) break;
                rem -= c;
            }
            const Inst& I = insts[q];
            if (I.sc->info) continue;
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= rem) ++a;
            const int b = rem - a * (a + 1) / 2;
            update_tile<T>(I, k, k + 1 + a, k + 1 + b, S1, S2);
        }
        if (!grid_barrier(bar, err)) return;
    }
}

// Solve L L' x = b for one right-hand side per instance (one CTA each).  The
// FP32 variant scales b by 1/||b||_inf so the working values stay O(1).
//
// Blocked substitution with 32-row blocks.  Warp 0 solves each 32 x 32
// diagonal block in registers (lane = row, shuffles carry the solved value);
// the other warps own the remaining rows and issue their 32 loads of the
// block's columns before waiting for the diagonal solve, so the L2 latency of
// the update overlaps the serial part.
template <typename T>
constexpr int solve_threads() { return sizeof(T) == 8 ? 256 : 512; }

template <typename T>
__global__ void __launch_bounds__(solve_threads<T>()) k_chol_solve(const Inst* __restrict__ insts, int in_role,
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
    const int nt = (n + kNb - 1) / kNb;
    // y holds nt*32 entries: the block updates read all 32 entries of the
    // last (short) block, whose tail stays zero.
    for (int j = threadIdx.x; j < nt * kNb; j += blockDim.x) y[j] = j < n ? (T)(bin[j] / sc) : T(0);
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nworkers = blockDim.x - 32, wid = threadIdx.x - 32;

    // ---- forward: L y = b
    for (int kb = 0; kb < nt; ++kb) {
        const int k0 = kb * kNb, kn = min(kNb, n - k0);
        if (warp == 0) {
            T Ld[kNb];
#pragma unroll
            for (int j = 0; j < kNb; ++j)
                Ld[j] = (lane < kn && j <= lane) ? L[(size_t)(k0 + lane) + (size_t)n * (k0 + j)] : T(0);
            T v = lane < kn ? y[k0 + lane] : T(0);
#pragma unroll
            for (int j = 0; j < kNb; ++j) {
                if (j < kn) {
                    T diag = __shfl_sync(full, Ld[j], j);
                    T yj = __shfl_sync(full, v, j) / diag;
                    if (lane == j) v = yj;
                    if (lane > j) v -= Ld[j] * yj;
                }
            }
            if (lane < kn) y[k0 + lane] = v;
        }
        // rows below the block: prefetch the block's columns, then wait for y_k
        for (int base = k0 + kn; base < n; base += nworkers) {
            const int i = base + wid;
            T Lr[kNb];
            if (warp > 0) {
#pragma unroll
                for (int j = 0; j < kNb; ++j) Lr[j] = (i < n && j < kn) ? L[(size_t)i + (size_t)n * (k0 + j)] : T(0);
            }
            if (base == k0 + kn) __syncthreads();   // y of this block is ready
            if (warp > 0 && i < n) {
                T acc = 0;
#pragma unroll
                for (int j = 0; j < kNb; ++j) acc += Lr[j] * y[k0 + j];
                y[i] -= acc;
            }
        }
        if (k0 + kn >= n) __syncthreads();
        __syncthreads();
    }
    // ---- backward: L' x = y
    for (int kb = nt - 1; kb >= 0; --kb) {
        const int k0 = kb * kNb, kn = min(kNb, n - k0);
        if (warp == 0) {
            T Lc[kNb];   // column 'lane' of the diagonal block: Lc[i] = L(k0+i, k0+lane)
#pragma unroll
            for (int i = 0; i < kNb; ++i)
                Lc[i] = (lane < kn && i < kn && i >= lane) ? L[(size_t)(k0 + i) + (size_t)n * (k0 + lane)] : T(0);
            T v = lane < kn ? y[k0 + lane] : T(0);
#pragma unroll
            for (int j = kNb - 1; j >= 0; --j) {
                if (j < kn) {
                    T diag = __shfl_sync(full, Lc[j], j);
                    T xj = __shfl_sync(full, v, j) / diag;
                    if (lane == j) v = xj;
                    if (lane < j) v -= Lc[j] * xj;
                }
            }
            if (lane < kn) y[k0 + lane] = v;
        }
        for (int base = 0; base < k0; base += nworkers) {
            const int i = base + wid;
            T Lr[kNb];   // Lr[j] = L(k0+j, i): row segment of column i
            if (warp > 0) {
#pragma unroll
                for (int j = 0; j < kNb; ++j) Lr[j] = (i < k0 && j < kn) ? L[(size_t)(k0 + j) + (size_t)n * i] : T(0);
            }
            if (base == 0) __syncthreads();
            if (warp > 0 && i < k0) {
                T acc = 0;
#pragma unroll
                for (int j = 0; j < kNb; ++j) acc += Lr[j] * y[k0 + j];
                y[i] -= acc;
            }
        }
        if (k0 == 0) __syncthreads();
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) xout[j] = (double)y[j] * sc;
}

// ---------------------------------------------------------------------------

void launch_potrf(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st) {
    static int occ[2] = {0, 0}, sms = 0;
    const int nt = (max_n + kNb - 1) / kNb;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_potrf_coop<float>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_potrf_coop<double>, 256, 0);
    }
    long long work = (long long)count * (nt * (nt + 1) / 2 > nt ? nt * (nt + 1) / 2 : nt);
    long long cap = (long long)occ[fp64 ? 1 : 0] * sms;
    int grid = (int)(work < cap ? work : cap);
    if (grid < 1) grid = 1;
    void* args[] = {(void*)&d_insts, (void*)&count, (void*)&nt, (void*)&flags};
    cudaError_t e;
    if (fp64)
        e = cudaLaunchCooperativeKernel((void*)k_potrf_coop<double>, dim3(grid), dim3(256), args, 0, st);
    else
        e = cudaLaunchCooperativeKernel((void*)k_potrf_coop<float>, dim3(grid), dim3(256), args, 0, st);
    note_launches(1);
    check_launch(st, e == cudaSuccess ? "k_potrf_coop" : "k_potrf_coop (launch refused)", __FILE__, __LINE__);
}

void launch_chol_solve(const Inst* d_insts, int count, int max_n, int fp64, int in_role,
                       int out_role, int flags, cudaStream_t st) {
    size_t smem = (size_t)((max_n + kNb - 1) / kNb) * kNb * (fp64 ? 8 : 4);
    if (fp64) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_chol_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(k_chol_solve<double><<<dim3(1, count), solve_threads<double>(), smem, st>>>(d_insts, in_role, out_role, flags));
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_chol_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(k_chol_solve<float><<<dim3(1, count), solve_threads<float>(), smem, st>>>(d_insts, in_role, out_role, flags));
    }
}

}  // namespace lqmpc
