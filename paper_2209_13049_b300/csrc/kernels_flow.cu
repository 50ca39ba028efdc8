// Dataflow Cholesky factorisation with the inverse of the factor (the FP32
// preconditioner of the mixed-precision solves, Eq. 7's M = L L') for one
// instance of n <= 544, one CTA per 32-wide block column.
//
// CTA j computes block column j of L one 32 x 32 row block p = j, j+1, ...
// at a time: L_pj = (A_pj - sum_{k<j} L_pk L_jk') L_jj^{-T}, the diagonal
// block factored and inverted in registers.  Every row block is published on
// its own (flag (j, p)), so CTA j+1 can factor its diagonal block as soon as
// L_{j+1,j} is out, while CTA j is still working down its column: the
// critical path is one diagonal factorisation plus two row blocks per block
// column.  Then CTA j forms block column j of X = L^{-1} by forward
// substitution down the column, X_pj = -X_pp sum_{k=j}^{p-1} L_pk X_kj,
// consuming row blocks as they appear (X_pp = L_pp^{-1} comes with flag (p, p)).
// The products sum over 32 k-columns per warp step in FP32 (the
// contraction is split over the eight warps and reduced in shared memory).
//
// Publication: a row block is written with L2-coherent stores, the CTA
// synchronises, and one thread sets its flag to the launch's epoch with a
// release store; readers poll the flags (bounded: a
// wait that gives up raises Scal::err bit 4 and the kernel still runs to its
// end) and read with L1-bypassing loads.  The epoch advances when the last
// CTA finishes, so flags never need clearing.  A non-positive pivot is
// recorded in Scal::info; every CTA still publishes, so nobody waits forever.
#include <algorithm>

#include "chol_diag.cuh"
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

namespace {

constexpr int kFb = 32;
constexpr int kFlowMaxN = 544;          // 17 block columns: the panels fit shared memory, 2 + 17^2 flags
constexpr uint32_t kFlowSpin = 1u << 22;

__device__ __forceinline__ int ld_flag(const int* p) { return *(const volatile int*)p; }

// Flag store with release semantics at GPU scope: the CTA's stores ordered
// before it (by the CTA barrier in front of it) are visible to whoever
// observes the flag and then acquires.
__device__ __forceinline__ void st_flag_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Flag load with acquire semantics at GPU scope: synchronises with the
// writer's release without a full fence (which would also wait for this
// thread's own outstanding stores).
__device__ __forceinline__ int ld_flag_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// 16-byte global -> shared copy through L2 only (other CTAs' data is read
// after their flag), zero-filled past `bytes` (0..16).
__device__ __forceinline__ void cpa16(float* dst, const float* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cpa_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Rows [32p, 32p + pr) of the global columns [mm0, mm1) of the column-major
// n x n matrix M into P[(mm - mmb) * 32 + r] (zeros for r >= pr) by the
// threads [t0, t0 + nthr): 16-byte copies when every column start is
// 16-byte aligned (n a multiple of 4), scalar L2 loads otherwise.  The
// copies are waited for by cpa_wait_all.
__device__ __forceinline__ void stage_rowblock(float* P, int mmb, const float* M, int n, int p, int pr, int mm0,
                                               int mm1, bool vec, int t0 = 0, int nthr = 256) {
    const int t = threadIdx.x - t0;
    if (vec) {
        for (int e = t; e < (mm1 - mm0) * 8; e += nthr) {
            const int mm = mm0 + e / 8, r = 4 * (e % 8);
            const int left = pr - r;
            const int bytes = left >= 4 ? 16 : (left > 0 ? 4 * left : 0);
            cpa16(P + (mm - mmb) * kFb + r, M + (size_t)n * mm + kFb * p + (left > 0 ? r : 0), bytes);
        }
    } else {
        for (int e = t; e < (mm1 - mm0) * kFb; e += nthr) {
            const int mm = mm0 + e / kFb, r = e % kFb;
            P[(mm - mmb) * kFb + r] = r < pr ? __ldcg(M + (size_t)n * mm + kFb * p + r) : 0.f;
        }
    }
}

// The CTA's own block A_pj (columns r0 .. r0 + kn - 1, rows p0 .. p0 + pr - 1
// of M, written by nobody else) into As column-major, zero-padded.
__device__ __forceinline__ void stage_own(float* As, const float* M, int n, int r0, int kn, int p0, int pr,
                                          bool vec, int t0 = 0, int nthr = 256) {
    const int t = threadIdx.x - t0;
    if (vec) {
        for (int e = t; e < kFb * 8; e += nthr) {
            const int c = e / 8, r = 4 * (e % 8), left = pr - r;
            if (c < kn) cpa16(As + c * kFb + r, M + (size_t)n * (r0 + c) + p0 + (left > 0 ? r : 0),
                              left >= 4 ? 16 : (left > 0 ? 4 * left : 0));
            else *reinterpret_cast<float4*>(As + c * kFb + r) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int e = t; e < kFb * kFb; e += nthr) {
            const int c = e / kFb, r = e % kFb;
            As[c * kFb + r] = (c < kn && r < pr) ? M[(size_t)n * (r0 + c) + p0 + r] : 0.f;
        }
    }
}

// Barrier of warps 1..7 (while warp 0 factors a diagonal block).
__device__ __forceinline__ void bar_w17() { asm volatile("bar.sync 1, 224;" ::: "memory"); }

// Warp W waits until the flags (k, p) for k in [k0, k1), and flag index
// `extra` when >= 0, all equal ep (one flag per lane, bounded); then the
// whole block (W = 0) or warps 1..7 (W = 1) proceed.
template <int W>
__device__ __forceinline__ void wait_flags(const int* flg, int nt, int k0, int k1, int p, int extra, int ep,
                                           int* err) {
    if ((threadIdx.x >> 5) == W) {
        const int lane = threadIdx.x & 31, cnt = k1 - k0;
        int idx = -1;
        if (lane < cnt) idx = (k0 + lane) * nt + p;
        else if (lane == cnt && extra >= 0) idx = extra;
        bool ok = idx < 0 || ld_flag_acquire(flg + idx) == ep;
        uint32_t it = 0;
        while (!__all_sync(0xffffffffu, ok)) {
            // give up after the bound, or soon after a wait anywhere gave up
            // (looked at every 64 polls, off the short waits' path)
            if ((++it & 63) == 0) {
                int stop = 0;
                if (lane == 0) stop = (it > kFlowSpin) || (ld_flag(err) & 4);
                if (__shfl_sync(0xffffffffu, stop, 0)) {
                    if (lane == 0) atomicOr(err, 4);
                    break;
                }
            }
            if (it > 256) __nanosleep(64);   // spin first: the wait is usually short
            if (!ok) ok = ld_flag_acquire(flg + idx) == ep;
        }
    }
    if (W == 0) __syncthreads();
    else bar_w17();
}

// acc[c] += sum_m P[m * 32 + lane] B[m * 32 + c] over m in [m0, m1), this
// warp (wi of nw) taking m = m0 + wi, m0 + wi + nw, ... (partial sums per warp).
__device__ __forceinline__ void acc_panel(float (&acc)[kFb], const float* P, const float* B, int m0, int m1,
                                          int wi = threadIdx.x >> 5, int nw = 8) {
    const int lane = threadIdx.x & 31;
    for (int m = m0 + wi; m < m1; m += nw) {
        const float a = P[m * kFb + lane];
        const float4* b4 = reinterpret_cast<const float4*>(B + m * kFb);
#pragma unroll
        for (int q = 0; q < kFb / 4; ++q) {
            const float4 b = b4[q];
            acc[4 * q + 0] = fmaf(a, b.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(a, b.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(a, b.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(a, b.w, acc[4 * q + 3]);
        }
    }
}

// Red[w][r][c] = warp w's partial (lane r); read back by reduce_into.
__device__ __forceinline__ void store_partial(const float (&acc)[kFb], float* Red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* R = Red + (warp * kFb + lane) * (kFb + 1);
#pragma unroll
    for (int c = 0; c < kFb; ++c) R[c] = acc[c];
}

__device__ __forceinline__ float sum_partials(const float* Red, int r, int c, int w0 = 0) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += w >= w0 ? Red[(w * kFb + r) * (kFb + 1) + c] : 0.f;
    return s;
}

// Warp 0: T (32 x 33, shared) -> L (D) and X = L^{-1} (Dv), lower, zeros
// above; returns 0, or q + 1 for the first non-positive pivot q.
//
// Left-looking by rounds of four columns, lane i holding row i of L in
// registers and every row also in shared memory: round j0 forms
// s_i,t = a_i,j0+t - sum_{k<j0} l_ik l_j0+t,k (rows j0..j0+3 read as
// broadcasts), takes the 4 x 4 pivot block from lanes j0..j0+3 by shuffles,
// factors it in every lane, and finishes the lane's four entries by
// substitution with it: one shared-memory exchange per four columns.  1/sqrt
// comes from rsqrtf refined by one Newton step, so the serial chain has no
// division.  The inverse by forward substitution L X = I with column `lane`
// of X in lane `lane`: x_i = (delta_{i,lane} - sum_{k<i} l_ik x_k) / l_ii.
// Not inlined, so its registers are allocated apart from the kernel's.
__device__ __noinline__ int factor_diag_block(const float* T, float* D, float* Dv) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __shared__ __align__(16) float Ls[kFb][kFb + 4];
    __shared__ float rs[kFb];
    float tr[kFb], l[kFb];
#pragma unroll
    for (int c = 0; c < kFb; ++c) tr[c] = T[lane * (kFb + 1) + c];
    int fail = 0;
    float rown = 1.f;
#pragma unroll
    for (int j0 = 0; j0 < kFb; j0 += 4) {
        float s[4][4];   // four partial sums per column
#pragma unroll
        for (int t = 0; t < 4; ++t) { s[t][0] = tr[j0 + t]; s[t][1] = s[t][2] = s[t][3] = 0.f; }
#pragma unroll
        for (int k4 = 0; k4 < j0 / 4; ++k4) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float4 lj = *reinterpret_cast<const float4*>(&Ls[j0 + t][4 * k4]);
                s[t][0] = fmaf(-l[4 * k4 + 0], lj.x, s[t][0]);
                s[t][1] = fmaf(-l[4 * k4 + 1], lj.y, s[t][1]);
                s[t][2] = fmaf(-l[4 * k4 + 2], lj.z, s[t][2]);
                s[t][3] = fmaf(-l[4 * k4 + 3], lj.w, s[t][3]);
            }
        }
        float sv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) sv[t] = (s[t][0] + s[t][1]) + (s[t][2] + s[t][3]);
        float P[4][4];   // pivot block, lower: P[t][u] = sv[u] of lane j0 + t
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int u = 0; u <= t; ++u) P[t][u] = __shfl_sync(full, sv[u], j0 + t);
        float B[4][4], rb[4];   // its factor and the reciprocals of the diagonal
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float d = P[t][t];
#pragma unroll
            for (int u = 0; u < t; ++u) d = fmaf(-B[t][u], B[t][u], d);
            const bool bad = !(d > 0.f);
            if (bad && !fail && lane == j0 + t) fail = j0 + t + 1;
            rb[t] = rsqrt_refined(bad ? 1.f : d);
            B[t][t] = d * rb[t];
#pragma unroll
            for (int v = t + 1; v < 4; ++v) {
                float e = P[v][t];
#pragma unroll
                for (int u = 0; u < t; ++u) e = fmaf(-B[v][u], B[t][u], e);
                B[v][t] = e * rb[t];
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float e = sv[t];
#pragma unroll
            for (int u = 0; u < t; ++u) e = fmaf(-l[j0 + u], B[t][u], e);
            const int col = j0 + t;
            l[col] = lane > col ? e * rb[t] : (lane == col ? B[t][t] : 0.f);
            if (lane == col) rown = rb[t];
        }
        *reinterpret_cast<float4*>(&Ls[lane][j0]) = make_float4(l[j0], l[j0 + 1], l[j0 + 2], l[j0 + 3]);
        __syncwarp();
    }
    rs[lane] = rown;
    __syncwarp();
    float x[kFb];
#pragma unroll
    for (int i = 0; i < kFb; ++i) {
        float v = i == lane ? 1.f : 0.f;
#pragma unroll
        for (int k4 = 0; k4 < (i + 3) / 4; ++k4) {
            const float4 li = *reinterpret_cast<const float4*>(&Ls[i][4 * k4]);
            if (4 * k4 + 0 < i) v = fmaf(-li.x, x[4 * k4 + 0], v);
            if (4 * k4 + 1 < i) v = fmaf(-li.y, x[4 * k4 + 1], v);
            if (4 * k4 + 2 < i) v = fmaf(-li.z, x[4 * k4 + 2], v);
            if (4 * k4 + 3 < i) v = fmaf(-li.w, x[4 * k4 + 3], v);
        }
        x[i] = v * rs[i];
    }
#pragma unroll
    for (int c = 0; c < kFb; ++c) {
        D[lane * (kFb + 1) + c] = l[c];
        Dv[c * (kFb + 1) + lane] = x[c];
    }
    const int f = __reduce_min_sync(full, fail ? fail : 0x7fffffff);
    return f == 0x7fffffff ? 0 : f;
}

}  // namespace

__global__ void __launch_bounds__(256, 1) k_potrf_flow(const Inst* __restrict__ insts, int flags) {
    pdl_wait();
    const Inst& I = insts[0];
    if (skip_instance(I, flags)) return;           // the same decision in every CTA
    extern __shared__ __align__(16) float fsm[];
    __shared__ float T[kFb][kFb + 1], D[kFb][kFb + 1], Dv[kFb][kFb + 1];
    __shared__ int ep_sh;
    const int n = I.n, nt = (n + kFb - 1) / kFb, j = blockIdx.x;
    int* epoch = I.pflags;        // [0] epoch, [1] finished CTAs, [2 + k nt + p] flag of row block p of column k
    int* done = I.pflags + 1;
    int* flg = I.pflags + 2;
    int* err = &I.sc->err;
    float* M = I.M32;
    if (threadIdx.x == 0) ep_sh = ld_flag(epoch) + 1;
    __syncthreads();
    const int ep = ep_sh;
    if (j >= nt) return;
    const int r0 = kFb * j, kn = min(kFb, n - r0);   // columns of this block column
    const int capP = max(j, nt - 1 - j);
    float* Rj = fsm;                                 // row block j of columns 0..r0-1: Rj[m * 32 + r] = L[r0 + r, m]
    float* Pn = Rj + kFb * kFb * j;                  // row block p of earlier columns, same layout
    float* Xs = Pn + kFb * kFb * capP;               // X[r0 + q, r0 + c] at Xs[q * 32 + c]
    float* As = Xs + kFb * kFb * (nt - j);           // A_pj, column-major
    float* Red = As + kFb * kFb;                     // [8 warps][32][33] partial sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (n % 4) == 0;
    if (j > 0 && warp == 0) {
        // Run the diagonal factorisation once on an identity block while
        // this CTA waits for its first columns anyway: its code (unrolled,
        // tens of KB) is then in the SM's instruction cache when the real
        // block arrives on the critical path.
        for (int e = lane; e < kFb * kFb; e += 32) T[e >> 5][e & 31] = (e >> 5) == (e & 31) ? 1.f : 0.f;
        __syncwarp();
        factor_diag_block(&T[0][0], &D[0][0], &Dv[0][0]);
    }

    // Row block p: A_pj into As and the partial sums of S = sum_{k<j} L_pk
    // L_jk' into Red (all warps); the last column's contribution comes last
    // (it is the latest to be published, on the critical path).
    auto gather = [&](int p) {
        const int p0 = kFb * p, pr = min(kFb, n - p0);
        float* P = p == j ? Rj : Pn;
        stage_own(As, M, n, r0, kn, p0, pr, vec);
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        if (j > 0) {
            const int kA = j - 1;
            if (kA > 0) {
                wait_flags<0>(flg, nt, 0, kA, p, -1, ep, err);
                stage_rowblock(P, 0, M, n, p, pr, 0, kFb * kA, vec);
                cpa_wait_all();
                __syncthreads();
                acc_panel(acc, P, Rj, 0, kFb * kA);
            }
            if (kA < j) {
                wait_flags<0>(flg, nt, j - 1, j, p, -1, ep, err);
                stage_rowblock(P, 0, M, n, p, pr, kFb * (j - 1), kFb * j, vec);
                cpa_wait_all();
                __syncthreads();
                acc_panel(acc, P, Rj, kFb * (j - 1), kFb * j);
            }
        }
        cpa_wait_all();
        store_partial(acc, Red);
        __syncthreads();
    };
    // T = A_pj - S from the partials of warps w0..7 (identity padding of a
    // ragged diagonal block)
    auto form_t = [&](bool diag, int w0) {
        for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
            const int r = e & 31, c = e >> 5;
            float v = As[c * kFb + r] - sum_partials(Red, r, c, w0);
            if (diag && r == c && r >= kn) v = 1.f;
            T[r][c] = v;
        }
        __syncthreads();
    };
    // L_pj = T X_jj' (lane -> row, warp -> 4 columns), stored to M
    auto solve_store = [&](int p) {
        const int p0 = kFb * p, pr = min(kFb, n - p0);
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int m = 0; m < kFb; ++m) {
            const float t = T[lane][m];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = fmaf(t, Dv[warp + 8 * q][m], o[q]);
        }
        if (lane < pr) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = warp + 8 * q;
                if (c < kn) __stcg(M + (size_t)n * (r0 + c) + p0 + lane, o[q]);
            }
        }
    };

    // diagonal block: warp 0 factors and inverts it (row i in lane i) while
    // warps 1..7 gather row block j+1, which then waits on nothing but this
    // factorisation; L_{j+1,j} goes out first (the next block column's
    // diagonal needs it), L_jj and X_jj with it
    gather(j);
    form_t(true, 0);
    const bool next = j + 1 < nt;
    if (warp == 0) {
        const int fail = factor_diag_block(&T[0][0], &D[0][0], &Dv[0][0]);
        if (lane == 0 && fail) atomicCAS(&I.sc->info, 0, r0 + fail);
    } else if (next) {
        const int q0 = r0 + kFb, qr = min(kFb, n - q0);
        stage_own(As, M, n, r0, kn, q0, qr, vec, 32, 224);
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        if (j > 1) {   // the columns published long ago, then the last one
            wait_flags<1>(flg, nt, 0, j - 1, j + 1, -1, ep, err);
            stage_rowblock(Pn, 0, M, n, j + 1, qr, 0, kFb * (j - 1), vec, 32, 224);
            cpa_wait_all();
            bar_w17();
            acc_panel(acc, Pn, Rj, 0, kFb * (j - 1), warp - 1, 7);
        }
        if (j > 0) {
            wait_flags<1>(flg, nt, j - 1, j, j + 1, -1, ep, err);
            stage_rowblock(Pn, 0, M, n, j + 1, qr, kFb * (j - 1), kFb * j, vec, 32, 224);
            cpa_wait_all();
            bar_w17();
            acc_panel(acc, Pn, Rj, kFb * (j - 1), kFb * j, warp - 1, 7);
        } else {
            cpa_wait_all();
        }
        store_partial(acc, Red);
    }
    __syncthreads();
    if (next) {
        form_t(false, 1);
        solve_store(j + 1);
        // L_{j+1,j} out before L_jj and X_jj: its release then waits on its
        // own stores only (the CTA barrier orders them before thread 0's
        // release)
        __syncthreads();
        if (threadIdx.x == 0) st_flag_release(flg + j * nt + j + 1, ep);
    }
    for (int c = warp; c < kn; c += 8) {
        if (lane < kn && lane >= c) {
            __stcg(M + (size_t)n * (r0 + c) + r0 + lane, D[lane][c]);
            const float xv = Dv[lane][c];
            __stcg(I.Xinv32 + (size_t)(r0 + lane) + (size_t)n * (r0 + c), xv);
            __stcg(I.XinvT32 + (size_t)(r0 + c) + (size_t)n * (r0 + lane), xv);
        }
    }
    for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) Xs[e] = Dv[e >> 5][e & 31];
    __syncthreads();
    if (threadIdx.x == 0) st_flag_release(flg + j * nt + j, ep);
    // the rest of the column
    for (int p = j + 2; p < nt; ++p) {
        gather(p);
        form_t(false, 0);
        solve_store(p);
        __syncthreads();
        if (threadIdx.x == 0) st_flag_release(flg + j * nt + p, ep);
    }

    // block column j of X: X_pj = -X_pp sum_{k=j}^{p-1} L_pk X_kj
    for (int p = j + 1; p < nt; ++p) {
        const int p0 = kFb * p, pr = min(kFb, n - p0);
        wait_flags<0>(flg, nt, j + 1, p, p, p * nt + p, ep, err);
        stage_rowblock(Pn, r0, M, n, p, pr, r0, p0, vec);
        for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
            const int r = e / kFb, c = e % kFb;   // X_pp[r][c]
            D[r][c] = (r < pr && c <= r) ? __ldcg(I.Xinv32 + (size_t)(p0 + r) + (size_t)n * (p0 + c)) : 0.f;
        }
        cpa_wait_all();
        __syncthreads();
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        acc_panel(acc, Pn, Xs, 0, p0 - r0);
        store_partial(acc, Red);
        __syncthreads();
        for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
            const int r = e & 31, c = e >> 5;
            T[r][c] = sum_partials(Red, r, c);
        }
        __syncthreads();
        // X_pj = -X_pp T: lane -> column, warp -> 4 rows
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int m = 0; m < kFb; ++m) {
            const float t = T[m][lane];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = fmaf(D[warp + 8 * q][m], t, o[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = warp + 8 * q;
            Xs[(p0 - r0 + r) * kFb + lane] = -o[q];
            if (r < pr && lane < kn) {
                I.Xinv32[(size_t)(p0 + r) + (size_t)n * (r0 + lane)] = -o[q];
                I.XinvT32[(size_t)(r0 + lane) + (size_t)n * (p0 + r)] = -o[q];
            }
        }
        __syncthreads();
    }
    // the last CTA to finish advances the epoch (every CTA has read it by
    // then; the next launch reads it after this one's end, so no fence)
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(done, 1) == nt - 1) {
        atomicExch(done, 0);
        atomicAdd(epoch, 1);
    }
}

// ---------------------------------------------------------------------------
// Queued dataflow Cholesky: any number of instances of n <= 1024 in one
// persistent cooperative launch (one CTA per SM).  The work is a list of
// tasks, per instance (largest first) the factor tasks of its block columns
// j = 0 .. nt-1 (L_pj for p >= j, as above, with X_jj) and then the inverse
// tasks j = 0 .. nt-2 (X_pj for p > j).  CTAs take tasks from a global
// ticket counter in list order.  A task waits only on the flags of tasks
// earlier in the list (a factor task on earlier block columns, an inverse
// task on factor tasks), and every earlier task has been taken by a
// resident CTA that does not wait on later ones, so every wait ends.  The
// earlier row blocks of L are staged through a chunk buffer of C blocks, so
// the shared memory holds one block row or column (nt blocks) plus a chunk.

namespace {

constexpr int kFlowQMaxN = 1024;        // 32 block columns: 2 + 32^2 flags, nt blocks of 32 x 32 per CTA

// acc += sum over block columns k in [k0, k1) of L(32p + lane, 32k + m)
// B[(32k + m) * 32 + c], the row block staged C block columns at a time
// through Pn after their flags (k, p); W = 0: all warps, W = 1: warps 1..7.
template <int W>
__device__ __forceinline__ void acc_rowblock(float (&acc)[kFb], float* Pn, int C, const float* B, const float* M,
                                             int n, const int* flg, int nt, int p, int pr, int k0, int k1, int ep,
                                             int* err, bool vec) {
    const int t0 = W ? 32 : 0, nthr = W ? 224 : 256;
    const int wi = (threadIdx.x >> 5) - (W ? 1 : 0), nw = W ? 7 : 8;
    for (int kc = k0; kc < k1; kc += C) {
        const int ke = min(k1, kc + C);
        // ends with a barrier of the participating warps: the previous chunk is consumed
        wait_flags<W>(flg, nt, kc, ke, p, -1, ep, err);
        stage_rowblock(Pn, kFb * kc, M, n, p, pr, kFb * kc, kFb * ke, vec, t0, nthr);
        cpa_wait_all();
        if (W) bar_w17();
        else __syncthreads();
        acc_panel(acc, Pn, B + kFb * kFb * kc, 0, kFb * (ke - kc), wi, nw);
    }
}

// T = A_pj - (sum of the partials of warps w0..7), identity padding of a
// ragged diagonal block
__device__ __forceinline__ void form_t_q(float (*T)[kFb + 1], const float* As, const float* Red, bool diag, int kn,
                                         int w0) {
    for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
        const int r = e & 31, c = e >> 5;
        float v = As[c * kFb + r] - sum_partials(Red, r, c, w0);
        if (diag && r == c && r >= kn) v = 1.f;
        T[r][c] = v;
    }
    __syncthreads();
}

// L_pj = T X_jj' (lane -> row, warp -> 4 columns), stored to M
__device__ __forceinline__ void solve_store_q(float (*T)[kFb + 1], float (*Dv)[kFb + 1], float* M, int n, int r0,
                                              int kn, int p) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p0 = kFb * p, pr = min(kFb, n - p0);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int m = 0; m < kFb; ++m) {
        const float t = T[lane][m];
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = fmaf(t, Dv[warp + 8 * q][m], o[q]);
    }
    if (lane < pr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = warp + 8 * q;
            if (c < kn) __stcg(M + (size_t)n * (r0 + c) + p0 + lane, o[q]);
        }
    }
}

struct FlowQSm {
    float* Big;    // nt blocks: row block j of the earlier columns (factor task), block column j of X (inverse task)
    float* Pn;     // C blocks: a chunk of an earlier row block of L
    float* As;     // A_pj, column-major
    float* Red;    // [8 warps][32][33] partial sums
    int C;
};

// Factor task of block column j of instance I.
__device__ __forceinline__ void flowq_factor(const Inst& I, int j, int ep, const FlowQSm& s, float (*T)[kFb + 1],
                                             float (*D)[kFb + 1], float (*Dv)[kFb + 1], bool warm) {
    const int n = I.n, nt = (n + kFb - 1) / kFb;
    const int r0 = kFb * j, kn = min(kFb, n - r0);
    int* flg = I.pflags + 2;
    int* err = &I.sc->err;
    float* M = I.M32;
    float* Rj = s.Big;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (n % 4) == 0;
    if (warm && j > 0 && warp == 0) {   // instruction-cache warm-up of the diagonal factorisation
        for (int e = lane; e < kFb * kFb; e += 32) T[e >> 5][e & 31] = (e >> 5) == (e & 31) ? 1.f : 0.f;
        __syncwarp();
        factor_diag_block(&T[0][0], &D[0][0], &Dv[0][0]);
    }
    // diagonal row block: row block j of columns 0..r0-1 into Rj (kept for
    // the whole task), the last column's part last
    {
        stage_own(s.As, M, n, r0, kn, r0, kn, vec);
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        if (j > 1) {
            wait_flags<0>(flg, nt, 0, j - 1, j, -1, ep, err);
            stage_rowblock(Rj, 0, M, n, j, kn, 0, kFb * (j - 1), vec);
            cpa_wait_all();
            __syncthreads();
            acc_panel(acc, Rj, Rj, 0, kFb * (j - 1));
        }
        if (j > 0) {
            wait_flags<0>(flg, nt, j - 1, j, j, -1, ep, err);
            stage_rowblock(Rj, 0, M, n, j, kn, kFb * (j - 1), kFb * j, vec);
            cpa_wait_all();
            __syncthreads();
            acc_panel(acc, Rj, Rj, kFb * (j - 1), kFb * j);
        }
        cpa_wait_all();
        store_partial(acc, s.Red);
        __syncthreads();
    }
    form_t_q(T, s.As, s.Red, true, kn, 0);
    // warp 0 factors and inverts the diagonal block while warps 1..7 gather
    // row block j+1; L_{j+1,j} goes out first (the next column's diagonal
    // waits for it), L_jj and X_jj with it
    const bool next = j + 1 < nt;
    if (warp == 0) {
        const int fail = factor_diag_block(&T[0][0], &D[0][0], &Dv[0][0]);
        if (lane == 0 && fail) atomicCAS(&I.sc->info, 0, r0 + fail);
    } else if (next) {
        const int q0 = r0 + kFb, qr = min(kFb, n - q0);
        stage_own(s.As, M, n, r0, kn, q0, qr, vec, 32, 224);
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        if (j > 1) acc_rowblock<1>(acc, s.Pn, s.C, Rj, M, n, flg, nt, j + 1, qr, 0, j - 1, ep, err, vec);
        if (j > 0) acc_rowblock<1>(acc, s.Pn, s.C, Rj, M, n, flg, nt, j + 1, qr, j - 1, j, ep, err, vec);
        cpa_wait_all();
        store_partial(acc, s.Red);
    }
    __syncthreads();
    if (next) {
        form_t_q(T, s.As, s.Red, false, kn, 1);
        solve_store_q(T, Dv, M, n, r0, kn, j + 1);
        __syncthreads();   // L_{j+1,j} out before L_jj and X_jj (a shorter release)
        if (threadIdx.x == 0) st_flag_release(flg + j * nt + j + 1, ep);
    }
    for (int c = warp; c < kn; c += 8) {
        if (lane < kn && lane >= c) {
            __stcg(M + (size_t)n * (r0 + c) + r0 + lane, D[lane][c]);
            const float xv = Dv[lane][c];
            __stcg(I.Xinv32 + (size_t)(r0 + lane) + (size_t)n * (r0 + c), xv);
            __stcg(I.XinvT32 + (size_t)(r0 + c) + (size_t)n * (r0 + lane), xv);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st_flag_release(flg + j * nt + j, ep);
    // the rest of the column
    for (int p = j + 2; p < nt; ++p) {
        const int p0 = kFb * p, pr = min(kFb, n - p0);
        stage_own(s.As, M, n, r0, kn, p0, pr, vec);
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        if (j > 1) acc_rowblock<0>(acc, s.Pn, s.C, Rj, M, n, flg, nt, p, pr, 0, j - 1, ep, err, vec);
        if (j > 0) acc_rowblock<0>(acc, s.Pn, s.C, Rj, M, n, flg, nt, p, pr, j - 1, j, ep, err, vec);
        cpa_wait_all();
        store_partial(acc, s.Red);
        __syncthreads();
        form_t_q(T, s.As, s.Red, false, kn, 0);
        solve_store_q(T, Dv, M, n, r0, kn, p);
        __syncthreads();
        if (threadIdx.x == 0) st_flag_release(flg + j * nt + p, ep);
    }
}

// Inverse task of block column j < nt-1: X_pj = -X_pp sum_{k=j}^{p-1} L_pk X_kj
// down the column, X_jj from the factor task's flag (j, j).
__device__ __forceinline__ void flowq_inverse(const Inst& I, int j, int ep, const FlowQSm& s, float (*T)[kFb + 1],
                                              float (*D)[kFb + 1]) {
    const int n = I.n, nt = (n + kFb - 1) / kFb;
    const int r0 = kFb * j;
    const int* flg = I.pflags + 2;
    int* err = &I.sc->err;
    const float* M = I.M32;
    float* Xs = s.Big;                  // X[r0 + q, r0 + c] at Xs[q * 32 + c]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool vec = (n % 4) == 0;
    wait_flags<0>(flg, nt, j, j + 1, j, -1, ep, err);
    for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {   // j < nt-1: a full block
        const int q = e >> 5, c = e & 31;
        Xs[e] = c <= q ? __ldcg(I.Xinv32 + (size_t)(r0 + q) + (size_t)n * (r0 + c)) : 0.f;
    }
    for (int p = j + 1; p < nt; ++p) {
        const int p0 = kFb * p, pr = min(kFb, n - p0);
        // L_pk for k in [j, p) and X_pp (flag (p, p)); ends with a barrier
        wait_flags<0>(flg, nt, j, p, p, p * nt + p, ep, err);
        for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
            const int r = e / kFb, c = e % kFb;
            D[r][c] = (r < pr && c <= r) ? __ldcg(I.Xinv32 + (size_t)(p0 + r) + (size_t)n * (p0 + c)) : 0.f;
        }
        float acc[kFb];
#pragma unroll
        for (int c = 0; c < kFb; ++c) acc[c] = 0.f;
        for (int kc = j; kc < p; kc += s.C) {
            const int ke = min(p, kc + s.C);
            if (kc > j) __syncthreads();   // the previous chunk is consumed
            stage_rowblock(s.Pn, kFb * kc, M, n, p, pr, kFb * kc, kFb * ke, vec);
            cpa_wait_all();
            __syncthreads();
            acc_panel(acc, s.Pn, Xs + kFb * kFb * (kc - j), 0, kFb * (ke - kc));
        }
        store_partial(acc, s.Red);
        __syncthreads();
        for (int e = threadIdx.x; e < kFb * kFb; e += blockDim.x) {
            const int r = e & 31, c = e >> 5;
            T[r][c] = sum_partials(s.Red, r, c);
        }
        __syncthreads();
        // X_pj = -X_pp T: lane -> column, warp -> 4 rows
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int m = 0; m < kFb; ++m) {
            const float t = T[m][lane];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = fmaf(D[warp + 8 * q][m], t, o[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = warp + 8 * q;
            Xs[(p0 - r0 + r) * kFb + lane] = -o[q];
            if (r < pr) {
                I.Xinv32[(size_t)(p0 + r) + (size_t)n * (r0 + lane)] = -o[q];
                I.XinvT32[(size_t)(r0 + lane) + (size_t)n * (p0 + r)] = -o[q];
            }
        }
        __syncthreads();
    }
}

}  // namespace

// tasks[t] = instance << 8 | kind << 7 | j (kind 0 factor, 1 inverse), in
// the order tickets are taken; ctl (2 words, zero between launches): ticket
// counter, exited CTAs.  Dynamic shared memory: (max_nt + C + 1) blocks of
// 32 x 32 and the partial sums.
__global__ void __launch_bounds__(256, 1) k_potrf_flowq(const Inst* __restrict__ insts, const int* __restrict__ tasks,
                                                        int ntasks, int max_nt, int C, int flags) {
    pdl_wait();
    extern __shared__ __align__(16) float fsm[];
    __shared__ float T[kFb][kFb + 1], D[kFb][kFb + 1], Dv[kFb][kFb + 1];
    __shared__ int task_sh, ep_sh;
    int* ctl = reinterpret_cast<int*>(insts[0].bar + 2);
    FlowQSm s;
    s.Big = fsm;
    s.Pn = s.Big + kFb * kFb * max_nt;
    s.As = s.Pn + kFb * kFb * C;
    s.Red = s.As + kFb * kFb;
    s.C = C;
    bool warm = true;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(ctl, 1);
            int task = t < ntasks ? tasks[t] : -1;
            if (task >= 0) {
                const Inst& I = insts[task >> 8];
                if (skip_instance(I, flags)) task = -2;
                else ep_sh = ld_flag(I.pflags) + 1;
            }
            task_sh = task;
        }
        __syncthreads();
        const int task = task_sh;
        const int ep = ep_sh;
        __syncthreads();
        if (task == -1) break;
        if (task == -2) continue;
        const Inst& I = insts[task >> 8];
        const int j = task & 127;
        if (task & 128) flowq_inverse(I, j, ep, s, T, D);
        else flowq_factor(I, j, ep, s, T, D, Dv, warm);
        warm = false;
        // the instance's last task to finish advances its epoch (every task
        // of it has read the epoch by then; later launches read it after this
        // one's end, so no fence)
        __syncthreads();
        if (threadIdx.x == 0) {
            const int nt = (I.n + kFb - 1) / kFb;
            if (atomicAdd(I.pflags + 1, 1) == 2 * nt - 2) {
                atomicExch(I.pflags + 1, 0);
                atomicAdd(I.pflags, 1);
            }
        }
    }
    // the last CTA out resets the ticket counter for the next launch
    if (threadIdx.x == 0 && atomicAdd(ctl + 1, 1) == (int)gridDim.x - 1) {
        atomicExch(ctl, 0);
        atomicExch(ctl + 1, 0);
    }
}


bool potrf_flowq_fits(int max_n) { return max_n >= 1 && max_n <= kFlowQMaxN; }

int flowq_task_count(int n) { return 2 * ((n + kFb - 1) / kFb) - 1; }

void flowq_tasks(int q, int n, int* out) {
    const int nt = (n + kFb - 1) / kFb;
    for (int j = 0; j < nt; ++j) *out++ = (q << 8) | j;
    for (int j = 0; j + 1 < nt; ++j) *out++ = (q << 8) | 128 | j;
}

bool launch_potrf_flowq(const Inst* d_insts, const int* d_tasks, int ntasks, int max_n, int flags, cudaStream_t st) {
    static int sms = 0, optin = 0, stat = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_potrf_flowq) == cudaSuccess) stat = (int)fa.sharedSizeBytes;
    }
    if (!potrf_flowq_fits(max_n) || !d_tasks || ntasks < 1) return false;
    const int nt = (max_n + kFb - 1) / kFb;
    const int blk = (int)sizeof(float) * kFb * kFb, red = (int)sizeof(float) * 8 * kFb * (kFb + 1);
    // the chunk: what is left after the block row / column and A_pj (at most nt blocks)
    const int C = std::min(nt, (optin - stat - red - (nt + 1) * blk) / blk);
    if (C < 1) return false;
    const size_t smem = (size_t)(nt + C + 1) * blk + red;
    if (cudaFuncSetAttribute(k_potrf_flowq, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_potrf_flowq, 256, smem);
    const int grid = std::min(ntasks, std::max(1, occ) * sms);
    int mnt = nt, c = C;
    void* args[] = {(void*)&d_insts, (void*)&d_tasks, (void*)&ntasks, (void*)&mnt, (void*)&c, (void*)&flags};
    cudaEvent_t pe = prof_start(st);
    // cooperative: every CTA is resident, so a task's waits on earlier tasks can end
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_potrf_flowq, dim3(grid), dim3(256), args, smem, st);
    note_launches(1);
    prof_stop(st, pe, "k_potrf_flowq");
    check_launch(st, "k_potrf_flowq", __FILE__, __LINE__);
    return e == cudaSuccess;
}

bool potrf_flow_fits(int count, int max_n) { return count == 1 && max_n >= 1 && max_n <= kFlowMaxN; }

bool launch_potrf_flow(const Inst* d_insts, int max_n, int flags, cudaStream_t st) {
    const int nt = (max_n + kFb - 1) / kFb;
    // per CTA j: j + max(j, nt-1-j) + (nt-j) + 1 blocks of 32 x 32, plus the partial sums
    int blocks = 0;
    for (int j = 0; j < nt; ++j) blocks = std::max(blocks, nt + std::max(j, nt - 1 - j) + 1);
    const size_t smem = sizeof(float) * ((size_t)blocks * kFb * kFb + 8 * kFb * (kFb + 1));
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
