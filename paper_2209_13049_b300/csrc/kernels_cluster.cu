// Cholesky factorisation of the condensed KKT matrix (Eq. 7) inside one
// thread-block cluster per instance, with the matrix held in the cluster's
// distributed shared memory.
//
// M (n <= 32 * kClMaxTiles) is cut into 32 x 32 tiles; lower tile (p, q)
// lives in the shared memory of CTA (p + q) mod kCl of the cluster.  Right-
// looking blocked Cholesky, per panel k:
//   (a) the owner of (k, k) factors it in registers (warp 0, shuffles) and
//       inverts the factor in the same sweep;
//   (b) panel tiles L_pk = A_pk L_kk^{-T} (p > k);
//   (c) trailing update A_pq -= L_pk L_qk^T (k < q <= p),
// separated by hardware cluster barriers; remote tiles are read over DSMEM.
// The FP32 variant also forms X = L^{-1} (the conjugate-gradient
// preconditioner) in the same loop by right-looking substitution on L X = I:
// X's row block k is L_kk^{-1} S_k* in step (b) and S_p* -= L_pk X_k* runs
// with step (c); S and X share storage.  A non-positive pivot stops the
// instance (Scal::info) without leaving any CTA waiting.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"
#include "chol_diag.cuh"

namespace cg = cooperative_groups;

namespace lqmpc {

constexpr int kCl = 8;            // CTAs per cluster
constexpr int kClNb = 32;         // tile edge
constexpr int kClLd = 33;         // padded row stride of a tile in shared memory
constexpr int kClMaxTiles = 16;   // tiles per side (n <= 512)
constexpr int kClMaxSlots = 18;   // most lower tiles any CTA owns for 16 tiles per side
constexpr int kClTile = kClNb * kClLd;

__host__ __device__ inline int cl_owner(int p, int q) { return (p + q) % kCl; }

// FP32 (with the inverse) also keeps a local copy of the panel column of the
// current step so the Schur updates read only local shared memory.
constexpr int kClCache = kClMaxTiles - 1;

template <typename T, bool INV>
constexpr size_t cluster_smem_bytes() {
    return (size_t)((INV ? 2 : 1) * kClMaxSlots + 3 + (INV ? kClCache : 0)) * kClTile * sizeof(T);
}

// C[r][c] (+)= sum_m A[r][m] B[c][m]   (A B^T), m < mlen (4 entries per thread)
template <typename T>
__device__ __forceinline__ void tile_abt(const T* A, const T* B, T acc[4]) {
    const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll 8
    for (int m = 0; m < kClNb; ++m) {
        const T a = A[r * kClLd + m];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] += a * B[(cb + 8 * e) * kClLd + m];
    }
}

// C[r][c] (+)= sum_m A[r][m] B[m][c]   (A B)
template <typename T>
__device__ __forceinline__ void tile_ab(const T* A, const T* B, T acc[4]) {
    const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll 8
    for (int m = 0; m < kClNb; ++m) {
        const T a = A[r * kClLd + m];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] += a * B[m * kClLd + cb + 8 * e];
    }
}

// Flat 16-byte copies of whole tiles (tiles are contiguous and 16-byte
// aligned); every load of a call is issued before its first store so remote
// (DSMEM) latency is paid once per call.
template <typename T>
__device__ __forceinline__ void tile_copy(T* dst, const T* src) {
    constexpr int NV = kClTile * (int)sizeof(T) / 16;
    constexpr int PER = (NV + 255) / 256;
    const float4* s = reinterpret_cast<const float4*>(src);
    float4* d = reinterpret_cast<float4*>(dst);
    float4 v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + 256 * i;
        if (e < NV) v[i] = s[e];
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + 256 * i;
        if (e < NV) d[e] = v[i];
    }
}

template <typename T>
__device__ __forceinline__ void tile_copy2(T* d0, const T* s0, T* d1, const T* s1) {
    constexpr int NV = kClTile * (int)sizeof(T) / 16;
    constexpr int PER = (NV + 255) / 256;
    const float4* a = reinterpret_cast<const float4*>(s0);
    const float4* b = reinterpret_cast<const float4*>(s1);
    float4 va[PER], vb[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + 256 * i;
        if (e < NV) { va[i] = a[e]; vb[i] = b[e]; }
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = threadIdx.x + 256 * i;
        if (e < NV) { reinterpret_cast<float4*>(d0)[e] = va[i]; reinterpret_cast<float4*>(d1)[e] = vb[i]; }
    }
}

template <typename T, bool INV>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(256, 1)
    k_potrf_cluster(const Inst* __restrict__ insts, int flags) {
    pdl_wait();
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const Inst& I = insts[blockIdx.x / kCl];
    // the same decision in every CTA of the cluster (flags do not change here)
    if (skip_instance(I, flags) || I.sc->info) return;
    extern __shared__ __align__(16) unsigned char cl_smem[];
    T* slotM = reinterpret_cast<T*>(cl_smem);
    T* slotX = slotM + (size_t)kClMaxSlots * kClTile;
    T* scr = slotM + (size_t)(INV ? 2 : 1) * kClMaxSlots * kClTile;   // 3 scratch tiles
    T* colc = scr + 3 * (size_t)kClTile;                               // panel-column cache (INV)
    __shared__ unsigned char slot_of[kClMaxTiles * (kClMaxTiles + 1) / 2];
    __shared__ int fail_sh;
    const int n = I.n, nt = (n + kClNb - 1) / kClNb;
    T* M = sizeof(T) == 8 ? (T*)I.M64 : (T*)I.M32;

    // tile -> slot table (same in every CTA)
    if (threadIdx.x == 0) {
        int cnt[kCl] = {0};
        for (int p = 0; p < nt; ++p)
            for (int q = 0; q <= p; ++q) {
                const int o = cl_owner(p, q);
                slot_of[p * (p + 1) / 2 + q] = (unsigned char)cnt[o]++;
            }
        fail_sh = 0;
    }
    __syncthreads();
    auto local_tile = [&](T* base, int p, int q) { return base + (size_t)slot_of[p * (p + 1) / 2 + q] * kClTile; };
    auto remote_tile = [&](T* base, int p, int q) {
        return cluster.map_shared_rank(local_tile(base, p, q), cl_owner(p, q));
    };

    // load the owned lower tiles; pad with the identity beyond n
    for (int p = 0; p < nt; ++p)
        for (int q = 0; q <= p; ++q) {
            if (cl_owner(p, q) != rank) continue;
            T* dst = local_tile(slotM, p, q);
            T* dx = INV ? local_tile(slotX, p, q) : nullptr;
            for (int e = threadIdx.x; e < kClNb * kClNb; e += blockDim.x) {
                const int r = e % kClNb, c = e / kClNb;
                const int gr = p * kClNb + r, gc = q * kClNb + c;
                T v = T(0);
                if (gr < n && gc < n) v = M[(size_t)gr + (size_t)n * gc];
                else if (gr == gc) v = T(1);
                dst[r * kClLd + c] = v;
                if (INV) dx[r * kClLd + c] = T(0);
            }
        }
    cluster.sync();

    int failed = 0;
    for (int k = 0; k < nt && !failed; ++k) {
        const int ok = cl_owner(k, k);
        // (a) diagonal factor and its inverse
        if (rank == ok) {
            T* D = local_tile(slotM, k, k);
            T* Dinv = INV ? local_tile(slotX, k, k) : scr + 2 * kClTile;
            // One warp, one row per lane.  Right-looking factorisation in
            // registers, then forward substitution L X = I with row i of X in
            // lane i's registers (X_j* = R_j* / l_jj, then R_i* -= l_ij X_j*
            // for i > j).
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                const unsigned full = 0xffffffffu;
                T a[kClNb];
#pragma unroll
                for (int c = 0; c < kClNb; ++c) a[c] = c <= lane ? D[lane * kClLd + c] : T(0);
                int fail = 0;
                T rdl = T(1);   // lane j: 1 / l_jj
#pragma unroll
                for (int j = 0; j < kClNb; ++j) {
                    if (!fail) {
                        const T djj = __shfl_sync(full, a[j], j);
                        if (!(djj > T(0))) {
                            fail = k * kClNb + j + 1;
                        } else {
                            T d, rd;
                            pivot_t<T>(djj, d, rd);
                            if (lane == j) rdl = rd;
                            const T lij = lane > j ? a[j] * rd : (lane == j ? d : T(0));
                            a[j] = lij;
#pragma unroll
                            for (int c = j + 1; c < kClNb; ++c) {
                                const T lcj = __shfl_sync(full, lij, c);
                                if (lane >= c) a[c] -= lij * lcj;
                            }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < kClNb; ++c) D[lane * kClLd + c] = c <= lane ? a[c] : T(0);
                __syncwarp();
                // forward substitution L X = I (L read back from shared memory)
                if (!fail) {
                    T x[kClNb];
#pragma unroll
                    for (int c = 0; c < kClNb; ++c) x[c] = c == lane ? T(1) : T(0);
#pragma unroll
                    for (int j = 0; j < kClNb; ++j) {
                        const T rd = __shfl_sync(full, rdl, j);
                        const T lij = D[lane * kClLd + j];
#pragma unroll
                        for (int c = 0; c < kClNb; ++c) {
                            if (c > j) break;
                            const T xjc = __shfl_sync(full, x[c], j) * rd;
                            x[c] = lane == j ? xjc : (lane > j ? x[c] - lij * xjc : x[c]);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < kClNb; ++c) Dinv[lane * kClLd + c] = c <= lane ? x[c] : T(0);
                }
                if (lane == 0) {
                    fail_sh = fail;
                    if (fail) atomicCAS(&I.sc->info, 0, fail);
                }
            }
        }
        cluster.sync();
        failed = *cluster.map_shared_rank(&fail_sh, ok);
        if (failed) break;
        // (b) panel tiles and X row block k
        {
            const T* DinvR = INV ? remote_tile(slotX, k, k)
                                 : cluster.map_shared_rank(scr + 2 * kClTile, ok);
            bool have = false;
            for (int p = k + 1; p < nt && !have; ++p) have = cl_owner(p, k) == rank;
            if (INV)
                for (int c = 0; c < k && !have; ++c) have = cl_owner(k, c) == rank;
            if (have) {
                tile_copy(scr, DinvR);     // scr[0] = L_kk^{-1}
                __syncthreads();
                for (int p = k + 1; p < nt; ++p) {
                    if (cl_owner(p, k) != rank) continue;
                    T* Apk = local_tile(slotM, p, k);
                    tile_copy(scr + kClTile, Apk);
                    __syncthreads();
                    T acc[4] = {0, 0, 0, 0};
                    tile_abt(scr + kClTile, scr, acc);      // A_pk L_kk^{-T}
                    const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll
                    for (int e = 0; e < 4; ++e) Apk[r * kClLd + cb + 8 * e] = acc[e];
                    __syncthreads();
                }
                if (INV)
                    for (int c = 0; c < k; ++c) {
                        if (cl_owner(k, c) != rank) continue;
                        T* Skc = local_tile(slotX, k, c);
                        tile_copy(scr + kClTile, Skc);
                        __syncthreads();
                        T acc[4] = {0, 0, 0, 0};
                        tile_ab(scr, scr + kClTile, acc);   // X_kc = L_kk^{-1} S_kc
                        const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll
                        for (int e = 0; e < 4; ++e) Skc[r * kClLd + cb + 8 * e] = acc[e];
                        __syncthreads();
                    }
            }
        }
        cluster.sync();
        // (c) trailing update of M, and of S (INV)
        if (INV) {
            // local copy of the panel column L_pk, p > k (batches of 4 tiles)
            bool need = false;
            for (int q = k + 1; q < nt && !need; ++q)
                for (int p = q; p < nt && !need; ++p) need = cl_owner(p, q) == rank;
            for (int p = k + 1; p < nt && !need; ++p)
                for (int c = 0; c <= k && !need; ++c) need = cl_owner(p, c) == rank;
            if (need) {
                for (int p = k + 1; p < nt; p += 2) {
                    if (p + 1 < nt)
                        tile_copy2(colc + (size_t)(p - k - 1) * kClTile, remote_tile(slotM, p, k),
                                   colc + (size_t)(p - k) * kClTile, remote_tile(slotM, p + 1, k));
                    else
                        tile_copy(colc + (size_t)(p - k - 1) * kClTile, remote_tile(slotM, p, k));
                }
                __syncthreads();
            }
            for (int q = k + 1; q < nt; ++q)
                for (int p = q; p < nt; ++p) {
                    if (cl_owner(p, q) != rank) continue;
                    T acc[4] = {0, 0, 0, 0};
                    tile_abt(colc + (size_t)(p - k - 1) * kClTile, colc + (size_t)(q - k - 1) * kClTile, acc);
                    T* Apq = local_tile(slotM, p, q);
                    const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll
                    for (int e = 0; e < 4; ++e) Apq[r * kClLd + cb + 8 * e] -= acc[e];
                }
            __syncthreads();
            for (int c = 0; c <= k; ++c) {
                bool mine = false;
                for (int p = k + 1; p < nt && !mine; ++p) mine = cl_owner(p, c) == rank;
                if (!mine) continue;
                tile_copy(scr, remote_tile(slotX, k, c));   // X_kc
                __syncthreads();
                for (int p = k + 1; p < nt; ++p) {
                    if (cl_owner(p, c) != rank) continue;
                    T acc[4] = {0, 0, 0, 0};
                    tile_ab(colc + (size_t)(p - k - 1) * kClTile, scr, acc);   // S_pc -= L_pk X_kc
                    T* Spc = local_tile(slotX, p, c);
                    const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll
                    for (int e = 0; e < 4; ++e) Spc[r * kClLd + cb + 8 * e] -= acc[e];
                }
                __syncthreads();
            }
        } else {
            for (int q = k + 1; q < nt; ++q)
                for (int p = q; p < nt; ++p) {
                    if (cl_owner(p, q) != rank) continue;
                    tile_copy2(scr, remote_tile(slotM, p, k), scr + kClTile, remote_tile(slotM, q, k));
                    __syncthreads();
                    T acc[4] = {0, 0, 0, 0};
                    tile_abt(scr, scr + kClTile, acc);
                    T* Apq = local_tile(slotM, p, q);
                    const int r = threadIdx.x % kClNb, cb = threadIdx.x / kClNb;
#pragma unroll
                    for (int e = 0; e < 4; ++e) Apq[r * kClLd + cb + 8 * e] -= acc[e];
                    __syncthreads();
                }
        }
        cluster.sync();
    }
    // write back L (and X, X^T) for the owned tiles
    if (!failed)
        for (int p = 0; p < nt; ++p)
            for (int q = 0; q <= p; ++q) {
                if (cl_owner(p, q) != rank) continue;
                const T* src = local_tile(slotM, p, q);
                const T* xs = INV ? local_tile(slotX, p, q) : nullptr;
                for (int e = threadIdx.x; e < kClNb * kClNb; e += blockDim.x) {
                    const int r = e % kClNb, c = e / kClNb;
                    const int gr = p * kClNb + r, gc = q * kClNb + c;
                    if (gr >= n || gc >= n || (p == q && c > r)) continue;
                    M[(size_t)gr + (size_t)n * gc] = src[r * kClLd + c];
                    if (INV) {
                        const float xv = (float)xs[r * kClLd + c];
                        I.Xinv32[(size_t)gr + (size_t)n * gc] = xv;
                        I.XinvT32[(size_t)gc + (size_t)n * gr] = xv;
                    }
                }
            }
    cluster.sync();   // no CTA leaves while its shared memory may still be read
}

bool potrf_cluster_fits(int max_n) { return (max_n + kClNb - 1) / kClNb <= kClMaxTiles; }

// Factor every instance with its own cluster when all fit (n <= 512).
bool launch_potrf_cluster(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st) {
    if ((max_n + kClNb - 1) / kClNb > kClMaxTiles) return false;
    cudaEvent_t pe = prof_start(st);
    cudaError_t e;
    if (fp64) {
        const size_t smem = cluster_smem_bytes<double, false>();
        cudaFuncSetAttribute(k_potrf_cluster<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_potrf_cluster<double, false><<<dim3(kCl * count), 256, smem, st>>>(d_insts, flags);
    } else {
        const size_t smem = cluster_smem_bytes<float, true>();
        cudaFuncSetAttribute(k_potrf_cluster<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_potrf_cluster<float, true><<<dim3(kCl * count), 256, smem, st>>>(d_insts, flags);
    }
    e = cudaGetLastError();
    note_launches(1);
    prof_stop(st, pe, fp64 ? "k_potrf_cluster<double>" : "k_potrf_cluster<float>");
    check_launch(st, "k_potrf_cluster", __FILE__, __LINE__);
    return e == cudaSuccess;
}

}  // namespace lqmpc
