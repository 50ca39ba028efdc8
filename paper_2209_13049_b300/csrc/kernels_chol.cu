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
#include "gamma_ff.cuh"
#include "chol_diag.cuh"

namespace lqmpc {

constexpr int kNb = 32;

template <typename T>
__device__ __forceinline__ T* kkt_mat(const Inst& I) {
    return sizeof(T) == 8 ? (T*)I.M64 : (T*)I.M32;
}

// Grid-wide barrier for the cooperative factorisation kernel (all CTAs are
// co-resident by the cooperative launch): thread 0 of each CTA arrives with an
// acquire-release add on the counter (its CTA's writes were ordered before it
// by the CTA barrier), the last one resets the counter and advances the
// generation word with a release add, the others poll the generation with
// acquire loads (spinning first, then sleeping between polls).  The spin is
// bounded: a barrier that gives up raises Scal::err bit 2 and lets the kernel
// return.
constexpr unsigned kBarLimit = 1u << 24;

__device__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived + 1u == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar), "r"(0u) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar + 1), "r"(1u) : "memory");
        } else {
            unsigned it = 0, cur;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar + 1) : "memory");
                if (cur != g) break;
                if (++it > kBarLimit) { ok = 0; atomicOr(err, 2); break; }
                if (it > 256) __nanosleep(32);
            }
        }
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
                    T d, rd;
                    pivot_t<T>(djj, d, rd);
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

// Inverse of the factored 32 x 32 diagonal block (lower triangular), one
// column per thread of warp 0, by forward substitution L x = e_c taken
// right-looking: once x_m is final it is subtracted from every later row at
// once (independent multiply-adds), so the dependent chain is two operations
// per row instead of a dot product per row (FP64 multiply-adds have a
// 64-cycle latency on this part).
template <typename T>
__device__ void invert_diag(T (*Ld)[kNb + 1], T (*Li)[kNb + 1]) {
    __shared__ T rd[kNb];
    if (threadIdx.x < kNb) rd[threadIdx.x] = T(1) / Ld[threadIdx.x][threadIdx.x];
    __syncthreads();
    if (threadIdx.x < kNb) {
        const int c = threadIdx.x;
        T x[kNb];
#pragma unroll
        for (int i = 0; i < kNb; ++i) x[i] = i == c ? T(1) : T(0);
#pragma unroll
        for (int m = 0; m < kNb; ++m) {
            if (m >= c) {
                x[m] *= rd[m];
#pragma unroll
                for (int i = m + 1; i < kNb; ++i) x[i] = fma_t<T>(-Ld[i][m], x[m], x[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < kNb; ++i) Li[i][c] = x[i];
    }
    __syncthreads();
}

// Panel k, row tile p.  Every CTA of the panel factors the diagonal block and
// inverts it; p == k writes L_kk (and L_kk^{-1} into the inverse when one is
// kept), p > k forms L_pk = A_pk L_kk^{-T} as a 32 x 32 x 32 product.
template <typename T>
__device__ void panel_tile(const Inst& I, int k, int p, T (*Ld)[kNb + 1], T (*Li)[kNb + 1], T (*A)[kNb + 1],
                           int* fail_sh, T* X) {
    T* M = kkt_mat<T>(I);
    const int n = I.n, k0 = k * kNb, kn = min(kNb, n - k0);
    if (!factor_diag<T>(I, M, k, p == k, Ld, fail_sh)) return;
    invert_diag<T>(Ld, Li);
    if (p == k) {
        // Other CTAs of this panel phase may still be reading A_kk from M to
        // factor it themselves, so L_kk is parked in ldiag[k % 2] and moved
        // into M by the diagonal CTA of the next panel phase (after the grid
        // barrier); the last panel has no other reader and writes M directly.
        const int nt = (n + kNb - 1) / kNb;
        T* park = reinterpret_cast<T*>(I.ldiag) + (size_t)(k % 2) * kNb * kNb;
        if (k > 0) {
            const T* prev = reinterpret_cast<const T*>(I.ldiag) + (size_t)((k - 1) % 2) * kNb * kNb;
            const int p0 = k0 - kNb;
            for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
                const int r = e % kNb, c = e / kNb;
                if (c <= r) M[(size_t)(p0 + r) + (size_t)n * (p0 + c)] = prev[e];
            }
        }
        for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
            const int r = e % kNb, c = e / kNb;
            if (r < kn && c < kn && c <= r) {
                if (k + 1 < nt) park[e] = Ld[r][c];
                else M[(size_t)(k0 + r) + (size_t)n * (k0 + c)] = Ld[r][c];
                if (X) {
                    X[(size_t)(k0 + r) + (size_t)n * (k0 + c)] = Li[r][c];
                    I.XinvT32[(size_t)(k0 + c) + (size_t)n * (k0 + r)] = (float)Li[r][c];
                }
            }
        }
        __syncthreads();
        return;
    }
    const int p0 = p * kNb;
    for (int e = threadIdx.x; e < kNb * kNb; e += blockDim.x) {
        const int r = e % kNb, c = e / kNb;
        A[r][c] = (p0 + r < n && c < kn) ? M[(size_t)(p0 + r) + (size_t)n * (k0 + c)] : T(0);
    }
    __syncthreads();
    // out[r][c] = sum_{m <= c} A[r][m] Li[c][m]: each thread's four entries
    // (row r, columns cb + 8q) as four interleaved chains
    {
        const int r = threadIdx.x % kNb, cb = threadIdx.x / kNb;   // 256 threads
        T acc[4] = {0, 0, 0, 0};
#pragma unroll 8
        for (int m = 0; m < kNb; ++m) {
            const T a = A[r][m];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (m <= cb + 8 * q) acc[q] = fma_t<T>(a, Li[cb + 8 * q][m], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = cb + 8 * q;
            if (p0 + r < n && c < kn) M[(size_t)(p0 + r) + (size_t)n * (k0 + c)] = acc[q];
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

// ---------------------------------------------------------------------------
// FP64 panel and update work.  An FP64 warp instruction holds one SM
// sub-partition's FP64 pipe for about 60 cycles on this part, so the layout
// above (one warp factors and inverts the 32 x 32 diagonal block, ~1000 FP64
// instructions on one sub-partition) took ~80 us per panel.  Here the factor
// runs on warps 0-3, one per sub-partition: warp w holds the columns
// c = w (mod 4), lane = row, and pivot j is taken by warp j % 4 as soon as
// column j has column j-1's update; the other warps wait for column j on a
// named barrier (producer bar.arrive, consumers bar.sync) while the producer
// goes on with its other columns.  Warps 4-7 take part in the same barriers
// and solve the panel's row tile against the columns as they appear
// (L_pk = A_pk L_kk^{-T} by right-looking substitution), so no inverse of the
// diagonal block is formed.

// d = sqrt(v), rd = 1/d: the FP32 seed r = rsqrtf(v) and one third-order
// step of the series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + O(e^3) with
// e = 1 - v r^2 (|e| <= 2^-21 from the seed, so the dropped terms are below
// 2^-62): three dependent FP64 operations instead of two Newton steps' six.
__device__ __forceinline__ void pivot64(double v, double& d, double& rd) {
    const float vf = (float)v;
    if (vf > 1e-30f && vf < 1e30f) {
        const double r = (double)rsqrtf(vf);
        const double e = fma(-v * r, r, 1.0);
        const double q = fma(0.375, e, 0.5);
        rd = fma(r * e, q, r);
        d = v * rd;
    } else {
        d = sqrt(v);
        rd = 1.0 / d;
    }
}

__device__ __forceinline__ void named_bar_sync256(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }
__device__ __forceinline__ void named_bar_arrive256(int id) { asm volatile("bar.arrive %0, 256;" ::"r"(id) : "memory"); }

// Warps 0-3: factor the diagonal block of panel k (rows/columns k0.., kn of
// them, identity padding) into Ld = L_kk (zero above the diagonal) and
// rdg = 1 / diag(L_kk), column j published on named barrier 1 + j % 4 (all
// 256 threads take part).  The first failing pivot (k0 + j + 1) goes to
// *fail_sh (zeroed by the caller); the steps after it go on (on NaNs) so that
// every barrier is met.  Barrier ids are reused every four steps: a warp
// can publish column j + 4 only after every warp has passed column j.
__device__ void factor_diag64(const double* M, int n, int k0, int kn, double (*Ld)[kNb + 1], double* rdg,
                              int* fail_sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double a[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int c = 4 * s + w;
        double v = (c == lane) ? 1.0 : 0.0;
        if (lane < kn && c < kn && c <= lane) v = M[(size_t)(k0 + lane) + (size_t)n * (k0 + c)];
        a[s] = v;
    }
    // column J of L from the owner's register a[J / 4]
#define LQ_PRODUCE64(J)                                                                   \
    {                                                                                     \
        const double djj = __shfl_sync(0xffffffffu, a[(J) >> 2], (J));                    \
        double d, rd;                                                                     \
        pivot64(djj, d, rd);                                                              \
        const bool bad = !(djj > 0.0);                                                    \
        const double l = lane > (J) ? a[(J) >> 2] * rd : (lane == (J) ? d : 0.0);         \
        a[(J) >> 2] = l;                                                                  \
        Ld[lane][(J)] = l;                                                                \
        if (lane == 0) {                                                                  \
            rdg[(J)] = rd;                                                                \
            if (bad && *fail_sh == 0) *fail_sh = k0 + (J) + 1;                            \
        }                                                                                 \
        __syncwarp();                                                                     \
        named_bar_arrive256(1 + ((J) & 3));                                               \
    }
    if (w == 0) LQ_PRODUCE64(0)
#pragma unroll
    for (int j = 0; j < kNb; ++j) {
        if (w != (j & 3)) named_bar_sync256(1 + (j & 3));
        const double li = Ld[lane][j];
        if (j + 1 < kNb && w == ((j + 1) & 3)) {
            a[(j + 1) >> 2] = fma(-li, Ld[j + 1][j], a[(j + 1) >> 2]);
            LQ_PRODUCE64(j + 1)
        }
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (4 * s + w > j + 1) a[s] = fma(-li, Ld[4 * s + w][j], a[s]);
    }
#undef LQ_PRODUCE64
}

// Panel k, row tile p, FP64: every CTA of the panel factors the diagonal
// block (warps 0-3); p == k stores L_kk (parked as in panel_tile); p > k has
// warps 4-7 solve X L_kk' = A_pk row by row while the columns of L_kk appear:
// lane = (row rho of the warp's 8, column class g = lane % 4) holds columns
// c = g (mod 4) of its row; at column j, x_j = a_j / L_jj is final and is
// subtracted, times L_cj, from every later column.
__device__ void panel_tile64(const Inst& I, int k, int p, double (*Ld)[kNb + 1], double* rdg, int* fail_sh) {
    double* M = I.M64;
    const int n = I.n, k0 = k * kNb, kn = min(kNb, n - k0), p0 = p * kNb;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) *fail_sh = 0;
    __syncthreads();
    const int g = lane & 3, r = 8 * (w - 4) + (lane >> 2);
    double x[8];
    if (w < 4) {
        factor_diag64(M, n, k0, kn, Ld, rdg, fail_sh);
    } else if (p == k) {
#pragma unroll
        for (int j = 0; j < kNb; ++j) named_bar_sync256(1 + (j & 3));
    } else {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int c = 4 * s + g;
            x[s] = (p0 + r < n && c < kn) ? M[(size_t)(p0 + r) + (size_t)n * (k0 + c)] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kNb; ++j) {
            named_bar_sync256(1 + (j & 3));
            const double xj = __shfl_sync(0xffffffffu, x[j >> 2], (lane & ~3) | (j & 3)) * rdg[j];
            // L_cj = 0 for c < j (groups with 4s + 3 < j are skipped whole);
            // c = j is overwritten by x_j below
#pragma unroll
            for (int s = 0; s < 8; ++s)
                if (4 * s + 3 >= j) x[s] = fma(-xj, Ld[4 * s + g][j], x[s]);
            if (g == (j & 3)) x[j >> 2] = xj;
        }
    }
    __syncthreads();
    const int fail = *fail_sh;
    if (fail) {
        if (p == k && tid == 0) atomicCAS(&I.sc->info, 0, fail);
        return;
    }
    if (p == k) {
        const int nt = (n + kNb - 1) / kNb;
        double* park = reinterpret_cast<double*>(I.ldiag) + (size_t)(k % 2) * kNb * kNb;
        if (k > 0) {
            const double* prev = reinterpret_cast<const double*>(I.ldiag) + (size_t)((k - 1) % 2) * kNb * kNb;
            const int q0 = k0 - kNb;
            for (int e = tid; e < kNb * kNb; e += blockDim.x) {
                const int rr = e % kNb, c = e / kNb;
                if (c <= rr) M[(size_t)(q0 + rr) + (size_t)n * (q0 + c)] = prev[e];
            }
        }
        for (int e = tid; e < kNb * kNb; e += blockDim.x) {
            const int rr = e % kNb, c = e / kNb;
            if (rr < kn && c < kn && c <= rr) {
                if (k + 1 < nt) park[e] = Ld[rr][c];
                else M[(size_t)(k0 + rr) + (size_t)n * (k0 + c)] = Ld[rr][c];
            }
        }
    } else if (w >= 4) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int c = 4 * s + g;
            if (p0 + r < n && c < kn) M[(size_t)(p0 + r) + (size_t)n * (k0 + c)] = x[s];
        }
    }
    __syncthreads();
}

// A_pq -= L_pk L_qk' on one 16 x 16 quadrant (quad = 2 * row half + column
// half) of the trailing tile (p, q), FP64: four work items per tile so that
// a panel's update spreads over four times as many SMs.  The quadrant above
// the diagonal of a diagonal tile is skipped.
__device__ void update_quad64(const Inst& I, int k, int p, int q, int quad, double (*Lp)[kNb + 1],
                              double (*Lq)[kNb + 1]) {
    double* M = I.M64;
    const int n = I.n, k0 = k * kNb, kn = min(kNb, n - k0);
    const int rh = quad >> 1, ch = quad & 1;
    if (p == q && rh < ch) return;
    const int r0 = p * kNb + 16 * rh, c0 = q * kNb + 16 * ch;
    for (int e = threadIdx.x; e < 16 * kNb; e += blockDim.x) {
        const int r = e % 16, c = e / 16;
        Lp[r][c] = (r0 + r < n && c < kn) ? M[(size_t)(r0 + r) + (size_t)n * (k0 + c)] : 0.0;
        Lq[r][c] = (c0 + r < n && c < kn) ? M[(size_t)(c0 + r) + (size_t)n * (k0 + c)] : 0.0;
    }
    __syncthreads();
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int c = 0; c < kNb; c += 2) {
        s0 = fma(Lp[ty][c], Lq[tx][c], s0);
        s1 = fma(Lp[ty][c + 1], Lq[tx][c + 1], s1);
    }
    const int row = r0 + ty, col = c0 + tx;
    if (row < n && col < n && col <= row) M[(size_t)row + (size_t)n * col] -= s0 + s1;
    __syncthreads();
}

// C (32 x 32 tile) = sum_{j in [j0, j1)} A_j B_j for tiles read from global
// column-major n x n matrices: A_j = tile (ar, j) of Amat, B_j = tile (j, bc)
// of Bmat (zero outside [0, n)).  The next pair of tiles is fetched into
// registers while the current pair is multiplied.  Result in registers
// (thread owns 4 entries: row threadIdx.x % 32, columns threadIdx.x / 32 + 8 e).
template <typename T>
__device__ void tile_chain(const T* Amat, const T* Bmat, int n, int ar, int bc, int j0, int j1,
                           T (*As)[kNb + 1], T (*Bs)[kNb + 1], T acc[4]) {
    const int r = threadIdx.x % kNb, cb = threadIdx.x / kNb;   // 256 threads: cb in 0..7
    T pa[4], pb[4];
    auto fetch = [&](int j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = cb + 8 * e;
            const int ra = ar * kNb + r, ca = j * kNb + c;
            const int rb = j * kNb + r, cbb = bc * kNb + c;
            pa[e] = (ra < n && ca < n) ? Amat[(size_t)ra + (size_t)n * ca] : T(0);
            pb[e] = (rb < n && cbb < n) ? Bmat[(size_t)rb + (size_t)n * cbb] : T(0);
        }
    };
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = 0;
    if (j0 >= j1) return;
    fetch(j0);
    for (int j = j0; j < j1; ++j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) { As[r][cb + 8 * e] = pa[e]; Bs[r][cb + 8 * e] = pb[e]; }
        __syncthreads();
        if (j + 1 < j1) fetch(j + 1);
#pragma unroll 8
        for (int m = 0; m < kNb; ++m) {
            const T a = As[r][m];
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[e] += a * Bs[m][cb + 8 * e];
        }
        __syncthreads();
    }
}

template <typename T>
__device__ void store_tile(T* Mat, int n, int tr, int tc, const T acc[4], T scale, T* MatT = nullptr) {
    const int r = threadIdx.x % kNb, cb = threadIdx.x / kNb;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int rr = tr * kNb + r, cc = tc * kNb + cb + 8 * e;
        if (rr < n && cc < n) {
            Mat[(size_t)rr + (size_t)n * cc] = scale * acc[e];
            if (MatT) MatT[(size_t)cc + (size_t)n * rr] = scale * acc[e];
        }
    }
}

// Right-looking blocked Cholesky of every participating instance in one
// cooperative launch: per panel, a panel phase (diagonal factor and inverse,
// panel product, one row tile per work item) and an update phase (one
// trailing tile per work item), separated by grid barriers.  Instances are
// chosen once at entry (not done, no earlier failure); a pivot failure only
// stops that instance's own work.
//
// With want_inv (the mixed-precision preconditioner) the kernel goes on to
// form X = L^{-1} by recursive 2 x 2 blocking over the 32-tiles: at level l
// (half size B = 2^l tiles) each pair of diagonal blocks [X11 0; X21 X22]
// gets X21 = -X22 (L21 X11), computed as T = L21 X11 then X21 = -X22 T (two
// barriered stages per level).  The diagonal tiles of X come from the panels.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf_coop(const Inst* __restrict__ insts, int count, int max_nt,
                                                    int flags, int want_inv) {
    pdl_wait();
    __shared__ T S1[kNb][kNb + 1];
    __shared__ T S2[kNb][kNb + 1];
    __shared__ T S3[kNb][kNb + 1];
    __shared__ T rdg[kNb];
    __shared__ int fail_sh;
    constexpr int kSub = sizeof(T) == 8 ? 4 : 1;   // update work items per trailing tile
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
            T* X = (want_inv && sizeof(T) == 4) ? (T*)I.Xinv32 : nullptr;
            if (I.sc->info) continue;
            if constexpr (sizeof(T) == 8)
                panel_tile64(I, k, k + rem, S1, rdg, &fail_sh);
            else
                panel_tile<T>(I, k, k + rem, S1, S2, S3, &fail_sh, X);
        }
        if (!grid_barrier(bar, err)) return;
        // update phase
        total = 0;
        for (int q = 0; q < count; ++q) {
            const Inst& I = insts[q];
            const int m = (I.n + kNb - 1) / kNb - k - 1;
            if (!skip_instance(I, flags) && m > 0) total += kSub * (m * (m + 1) / 2);
        }
        for (int item = blockIdx.x; item < total; item += gridDim.x) {
            int q = 0, rem = item;
            for (;; ++q) {
                const Inst& I = insts[q];
                const int m = (I.n + kNb - 1) / kNb - k - 1;
                const int c = (!skip_instance(I, flags) && m > 0) ? kSub * (m * (m + 1) / 2) : 0;
                if (rem < c) break;
                rem -= c;
            }
            const Inst& I = insts[q];
            if (I.sc->info) continue;
            const int sub = rem % kSub;
            rem /= kSub;
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= rem) ++a;
            const int b = rem - a * (a + 1) / 2;
            if constexpr (sizeof(T) == 8)
                update_quad64(I, k, k + 1 + a, k + 1 + b, sub, S1, S2);
            else
                update_tile<T>(I, k, k + 1 + a, k + 1 + b, S1, S2);
        }
        if (!grid_barrier(bar, err)) return;
    }
    if (!want_inv || sizeof(T) != 4) return;
    // ---- X = L^{-1} by recursive doubling over the 32-tiles
    for (int B = 1; B < max_nt; B <<= 1) {
        for (int stage = 0; stage < 2; ++stage) {
            // tasks: for each instance, each pair i (lo1 = 2 i B), each tile (p, c),
            // p in [lo1 + B, min(lo1 + 2B, nt)), c in [lo1, lo1 + B)
            int total = 0;
            for (int q = 0; q < count; ++q) {
                const Inst& I = insts[q];
                if (skip_instance(I, flags)) continue;
                const int nt = (I.n + kNb - 1) / kNb;
                for (int lo1 = 0; lo1 + B < nt; lo1 += 2 * B) total += B * (min(lo1 + 2 * B, nt) - lo1 - B);
            }
            for (int item = blockIdx.x; item < total; item += gridDim.x) {
                int q = 0, rem = item, lo1 = 0, np = 0;
                bool found = false;
                for (; q < count && !found; ++q) {
                    const Inst& I = insts[q];
                    if (skip_instance(I, flags)) continue;
                    const int nt = (I.n + kNb - 1) / kNb;
                    for (lo1 = 0; lo1 + B < nt; lo1 += 2 * B) {
                        np = min(lo1 + 2 * B, nt) - lo1 - B;
                        if (rem < B * np) { found = true; break; }
                        rem -= B * np;
                    }
                    if (found) break;
                }
                const Inst& I = insts[q];
                if (I.sc->info) continue;
                const int p = lo1 + B + rem / B, c = lo1 + rem % B;
                const float* L = I.M32;
                float* X = I.Xinv32;
                float* Tm = I.Tinv32;
                T acc[4];
                if (stage == 0) {   // T_pc = sum_{j = c}^{lo1 + B - 1} L_pj X_jc
                    tile_chain<T>((const T*)L, (const T*)X, I.n, p, c, c, lo1 + B, S1, S2, acc);
                    store_tile<T>((T*)Tm, I.n, p, c, acc, T(1));
                } else {            // X_pc = -sum_{j = lo1 + B}^{p} X_pj T_jc
                    tile_chain<T>((const T*)X, (const T*)Tm, I.n, p, c, lo1 + B, p + 1, S1, S2, acc);
                    store_tile<T>((T*)X, I.n, p, c, acc, T(-1), (T*)I.XinvT32);
                }
            }
            if (!grid_barrier(bar, err)) return;
        }
    }
}

// Preconditioner of the mixed-precision conjugate gradients: z = X' (X r)
// with X = L^{-1} (FP32, lower).  Stage 1: t = X r, row by row (rows of X
// are the contiguous columns of X'); stage 2: z = X' t, column by column.
//
// The two-level tier's combined inverse Y is held as hi + lo planes
// (Xinv32 + Xlo32, transposes likewise) and applied with float-float sums:
// t = Y r (t as hi + lo), z = Y' t.
__device__ __forceinline__ void ffp_mac(float& sh, float& sl, float xh, float xl, float vh, float vl) {
    const float p = xh * vh;
    float e = fmaf(xh, vh, -p);
    e = fmaf(xh, vl, e);
    e = fmaf(xl, vh, e);
    const float s = sh + p;
    const float z = s - sh;
    sl += ((sh - (s - z)) + (p - z)) + e;
    sh = s;
}
__device__ __forceinline__ void ffp_warp_sum(float& sh, float& sl) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
        const float s = sh + oh;
        const float z = s - sh;
        sl += ((sh - (s - z)) + (oh - z)) + ol;
        sh = s;
    }
}

// Four warps per CTA, WPR warps per row (k_prec_lower) or column
// (k_prec_upper): a single instance takes a whole CTA per row (WPR = 4, its
// loads in flight at once for n <= 512, the warps' sums met in shared
// memory), a batch one warp per row (WPR = 1, four rows per CTA).
constexpr int kPrecThreads = 128, kPrecU = 4;

// The row group of the calling thread: group g, thread tg of GT.
template <int WPR>
struct PrecGroup {
    static constexpr int RPC = kPrecThreads / 32 / WPR, GT = 32 * WPR;
    int g, tg;
    __device__ PrecGroup() : g((threadIdx.x >> 5) / WPR), tg(threadIdx.x % (32 * WPR)) {}
};

// FP32 dot of a and x over len entries (FP64 x cast to FP32), the group's
// sum in its thread 0 (tg == 0).  Every thread of the CTA calls it (len 0
// for a group without a row).
template <int WPR, typename TX>
__device__ __forceinline__ float prec_dot32(const float* a, const TX* x, int len, float* wsum) {
    const PrecGroup<WPR> G;
    float av[kPrecU], xv[kPrecU];
#pragma unroll
    for (int u = 0; u < kPrecU; ++u) {
        const int e = G.tg + G.GT * u;
        av[u] = e < len ? a[e] : 0.f;
        xv[u] = e < len ? (float)x[e] : 0.f;
    }
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < kPrecU; ++u) acc = fmaf(av[u], xv[u], acc);
    for (int e = G.tg + G.GT * kPrecU; e < len; e += G.GT) acc = fmaf(a[e], (float)x[e], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (WPR > 1) {
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (G.tg == 0) {
            acc = 0.f;
#pragma unroll
            for (int w = 0; w < WPR; ++w) acc += wsum[G.g * WPR + w];
        }
        __syncthreads();
    }
    return acc;
}

// The same in float-float: a = ah + al, x = xh + xl (x given as FP64 when
// xd); the group's sum (oh, ol) in its thread 0.
template <int WPR>
__device__ __forceinline__ void prec_dot_ff(const float* ah, const float* al, const double* xd, const float* xh,
                                            const float* xl, int len, float* wsh, float* wsl, float& oh, float& ol) {
    const PrecGroup<WPR> G;
    float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f};
    auto mac = [&](int e, float& h, float& l) {
        float vh, vl;
        if (xd) { vh = (float)xd[e]; vl = (float)(xd[e] - (double)vh); }
        else { vh = xh[e]; vl = xl[e]; }
        ffp_mac(h, l, ah[e], al[e], vh, vl);
    };
    for (int e = G.tg; e < len; e += 2 * G.GT) {   // two independent chains
        mac(e, sh[0], sl[0]);
        if (e + G.GT < len) mac(e + G.GT, sh[1], sl[1]);
    }
    ffp_warp_sum(sh[0], sl[0]);
    ffp_warp_sum(sh[1], sl[1]);
    {
        const float s = sh[0] + sh[1], z = s - sh[0];
        sl[0] = ((sh[0] - (s - z)) + (sh[1] - z)) + sl[0] + sl[1];
        sh[0] = s;
    }
    oh = sh[0]; ol = sl[0];
    if (WPR > 1) {
        if ((threadIdx.x & 31) == 0) { wsh[threadIdx.x >> 5] = sh[0]; wsl[threadIdx.x >> 5] = sl[0]; }
        __syncthreads();
        if (G.tg == 0) {
            float h = wsh[G.g * WPR], l = wsl[G.g * WPR];
            for (int w = 1; w < WPR; ++w) {
                const float hw = wsh[G.g * WPR + w];
                const float s = h + hw, z = s - h;
                l += ((h - (s - z)) + (hw - z)) + wsl[G.g * WPR + w];
                h = s;
            }
            oh = h; ol = l;
        }
        __syncthreads();
    }
}

template <int WPR>
__global__ void __launch_bounds__(kPrecThreads) k_prec_lower(const Inst* __restrict__ insts, int in_role, int flags) {
    pdl_wait();
    __shared__ float wsh[kPrecThreads / 32], wsl[kPrecThreads / 32];
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    const double* r = role_ptr(I, in_role);
    const int n = I.n;
    const PrecGroup<WPR> G;
    const float* XT = I.XinvT32;   // X' column-major: row i of X is contiguous
    const bool two = I.sc->prec_cur == kPrecTwoLevel;
    for (int i0 = blockIdx.x * G.RPC; i0 < n; i0 += gridDim.x * G.RPC) {   // uniform trip count in the CTA
        const int i = i0 + G.g, len = i < n ? i + 1 : 0;
        const size_t ro = (size_t)n * (i < n ? i : 0);
        if (two) {
            float h, l;
            prec_dot_ff<WPR>(XT + ro, I.XloT32 + ro, r, nullptr, nullptr, len, wsh, wsl, h, l);
            if (G.tg == 0 && i < n) {
                I.r32[i] = h + l;
                I.r32lo[i] = l - ((h + l) - h);
            }
        } else {
            const float acc = prec_dot32<WPR>(XT + ro, r, len, wsh);
            if (G.tg == 0 && i < n) I.r32[i] = acc;
        }
    }
}

// tail (conjugate-gradient direction from z, run by the instance's last CTA):
// 1 p = z and r'z; 2 beta = r'z_new / r'z_old, p = z + beta p, either split
// for the next float-float Gamma p.  Tail 3 only splits z itself, element by
// element (the float-float Gamma du that follows the first solve).
template <int WPR>
__global__ void __launch_bounds__(kPrecThreads) k_prec_upper(const Inst* __restrict__ insts, int out_role, int flags,
                                                             int tail) {
    pdl_wait();
    __shared__ double red[32];
    __shared__ double beta_sh;
    __shared__ float wsh[kPrecThreads / 32], wsl[kPrecThreads / 32];
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    double* z = role_ptr(I, out_role);
    const int n = I.n;
    const PrecGroup<WPR> G;
    const float* X = I.Xinv32;
    const bool two = I.sc->prec_cur == kPrecTwoLevel;
    for (int j0 = blockIdx.x * G.RPC; j0 < n; j0 += gridDim.x * G.RPC) {   // uniform trip count in the CTA
        const int j = j0 + G.g, jj = j < n ? j : 0, len = j < n ? n - j : 0;
        const size_t c0 = (size_t)n * jj + jj;    // column j from row j on
        double zj;
        if (two) {
            float h, l;
            prec_dot_ff<WPR>(X + c0, I.Xlo32 + c0, nullptr, I.r32 + jj, I.r32lo + jj, len, wsh, wsl, h, l);
            zj = (double)h + (double)l;
        } else {
            zj = (double)prec_dot32<WPR>(X + c0, I.r32 + jj, len, wsh);
        }
        if (G.tg == 0 && j < n) {
            z[j] = zj;
            if (tail == 3) split_ff(zj, I.ffv[j], I.ffv[n + j]);
        }
    }
    if ((tail != 1 && tail != 2) || !last_arrival(I.sc)) return;
    Scal* S = I.sc;
    double rz = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) rz += I.rho[k] * __ldcg(z + k);
    rz = block_reduce<0>(rz, red);
    if (threadIdx.x == 0) {
        beta_sh = (tail == 2 && S->pcg_rz != 0.0) ? rz / S->pcg_rz : 0.0;
        S->pcg_rz = rz;
    }
    __syncthreads();
    const double be = beta_sh;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double pk = __ldcg(z + k) + (be != 0.0 ? be * I.pp[k] : 0.0);
        I.pp[k] = pk;
        split_ff(pk, I.ffv[k], I.ffv[n + k]);   // the next float-float Gamma p needs no split launch
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
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* y = (T*)smem_raw;
    __shared__ double red[32];
    // y: nt*32 entries, then the reciprocals of L's diagonal (nt*32)
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
    // reciprocals of the diagonal up front (in parallel): the substitution
    // chains then multiply instead of divide (an FP64 division takes ~430
    // cycles of latency on this part, a multiply 64)
    T* rdiag = y + nt * kNb;
    for (int j = threadIdx.x; j < nt * kNb; j += blockDim.x) {
        y[j] = j < n ? (T)(bin[j] / sc) : T(0);
        rdiag[j] = j < n ? T(1) / L[(size_t)j + (size_t)n * j] : T(1);
    }
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nworkers = blockDim.x - 32, wid = threadIdx.x - 32;

    // ---- forward: L y = b.  Warp 0 holds the current diagonal block in Ld
    // and loads the next one while the other warps apply the update.
    T Ld[kNb];
    if (warp == 0) {
        const int kn0 = min(kNb, n);
#pragma unroll
        for (int j = 0; j < kNb; ++j) Ld[j] = (lane < kn0 && j <= lane) ? L[(size_t)lane + (size_t)n * j] : T(0);
    }
    for (int kb = 0; kb < nt; ++kb) {
        const int k0 = kb * kNb, kn = min(kNb, n - k0);
        if (warp == 0) {
            T v = lane < kn ? y[k0 + lane] : T(0);
            const T rl = rdiag[k0 + lane];
#pragma unroll
            for (int j = 0; j < kNb; ++j) {
                if (j < kn) {
                    const T yj = __shfl_sync(full, v * rl, j);
                    if (lane == j) v = yj;
                    if (lane > j) v -= Ld[j] * yj;
                }
            }
            if (lane < kn) y[k0 + lane] = v;
            if (kb + 1 < nt) {   // prefetch the next diagonal block
                const int k1 = k0 + kNb, kn1 = min(kNb, n - k1);
#pragma unroll
                for (int j = 0; j < kNb; ++j)
                    Ld[j] = (lane < kn1 && j <= lane) ? L[(size_t)(k1 + lane) + (size_t)n * (k1 + j)] : T(0);
            }
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
                T acc[4] = {0, 0, 0, 0};   // four independent chains
#pragma unroll
                for (int j = 0; j < kNb; ++j) acc[j & 3] += Lr[j] * y[k0 + j];
                y[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
            }
        }
        if (k0 + kn >= n) __syncthreads();
        __syncthreads();
    }
    // ---- backward: L' x = y (columns of the diagonal block, prefetched likewise)
    if (warp == 0) {
        const int k0 = (nt - 1) * kNb, kn = n - k0;
#pragma unroll
        for (int i = 0; i < kNb; ++i)
            Ld[i] = (lane < kn && i < kn && i >= lane) ? L[(size_t)(k0 + i) + (size_t)n * (k0 + lane)] : T(0);
    }
    for (int kb = nt - 1; kb >= 0; --kb) {
        const int k0 = kb * kNb, kn = min(kNb, n - k0);
        if (warp == 0) {
            T v = lane < kn ? y[k0 + lane] : T(0);
            const T rl = rdiag[k0 + lane];
#pragma unroll
            for (int j = kNb - 1; j >= 0; --j) {
                if (j < kn) {
                    const T xj = __shfl_sync(full, v * rl, j);
                    if (lane == j) v = xj;
                    if (lane < j) v -= Ld[j] * xj;
                }
            }
            if (lane < kn) y[k0 + lane] = v;
            if (kb > 0) {   // prefetch the previous block's diagonal columns (full block)
                const int km = k0 - kNb;
#pragma unroll
                for (int i = 0; i < kNb; ++i)
                    Ld[i] = (i >= lane) ? L[(size_t)(km + i) + (size_t)n * (km + lane)] : T(0);
            }
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
                T acc[4] = {0, 0, 0, 0};
#pragma unroll
                for (int j = 0; j < kNb; ++j) acc[j & 3] += Lr[j] * y[k0 + j];
                y[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
            }
        }
        if (k0 == 0) __syncthreads();
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) xout[j] = (double)y[j] * sc;
}

// ---------------------------------------------------------------------------

void launch_potrf(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st, int want_inv,
                  int variant, const int* d_tasks, int ntasks) {
    static int occ[2] = {0, 0}, sms = 0;
    const int nt = (max_n + kNb - 1) / kNb;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_potrf_coop<float>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_potrf_coop<double>, 256, 0);
    }
    // variant: -1 the rule below, 0 cooperative, 1 clusters where they apply
    // (in a batch with instances over the cluster limit: clusters for the
    // others, then the queued dataflow kernel -- or the cooperative one past
    // its limit -- for those), 2 dataflow (one instance of n <= 544: one CTA
    // per block column; otherwise the queued kernel), 3 the queued kernel --
    // autotuned.  The rule: FP32 with the inverse takes the dataflow kernels
    // (one instance: measured 0.20 ms for n = 500 against 0.37-0.50 ms
    // cooperative and 0.53 ms in a cluster), except that a batch filling the
    // GPU with one 8-CTA cluster per instance factors its small instances in
    // clusters; FP64 takes clusters for such batches and the cooperative
    // kernel otherwise (its pipe rate makes 8 SMs too few for one instance).
    const bool dataflow = !fp64 && want_inv;
    const bool flowq_ok = dataflow && d_tasks && potrf_flowq_fits(max_n);
    const bool want_cluster = variant == 1 || (variant < 0 && count * 8 >= sms);
    if (dataflow && (variant == 2 || (variant < 0 && !want_cluster)) && potrf_flow_fits(count, max_n) &&
        launch_potrf_flow(d_insts, max_n, flags, st))
        return;
    if (flowq_ok && (variant == 2 || variant == 3 || (variant < 0 && !want_cluster)) &&
        launch_potrf_flowq(d_insts, d_tasks, ntasks, max_n, flags, st))
        return;
    const bool cluster_ok = fp64 || want_inv;
    if (cluster_ok && want_cluster && launch_potrf_cluster(d_insts, count, max_n, fp64, flags, st)) return;
    if (cluster_ok && want_cluster && count > 1 && launch_potrf_cluster(d_insts, count, 512, fp64, flags | F_N_LE_512, st)) {
        flags |= F_N_GT_512;   // the small instances are factored; the rest follow
        if (flowq_ok && launch_potrf_flowq(d_insts, d_tasks, ntasks, max_n, flags, st)) return;
    }
    long long work = (long long)count * (nt * (nt + 1) / 2 > nt ? nt * (nt + 1) / 2 : nt) * (fp64 ? 4 : 1);
    // FP64: one CTA per SM, so that the panel's CTAs (each factoring the
    // diagonal block on four sub-partitions' FP64 pipes) never share an SM
    long long cap = fp64 ? (long long)sms : (long long)occ[0] * sms;
    int grid = (int)(work < cap ? work : cap);
    if (grid < 1) grid = 1;
    void* args[] = {(void*)&d_insts, (void*)&count, (void*)&nt, (void*)&flags, (void*)&want_inv};
    cudaEvent_t pe = prof_start(st);
    cudaError_t e;
    if (fp64)
        e = cudaLaunchCooperativeKernel((void*)k_potrf_coop<double>, dim3(grid), dim3(256), args, 0, st);
    else
        e = cudaLaunchCooperativeKernel((void*)k_potrf_coop<float>, dim3(grid), dim3(256), args, 0, st);
    note_launches(1);
    prof_stop(st, pe, fp64 ? "k_potrf_coop<double>" : "k_potrf_coop<float>");
    check_launch(st, e == cudaSuccess ? "k_potrf_coop" : "k_potrf_coop (launch refused)", __FILE__, __LINE__);
}

void launch_prec_apply(const Inst* d_insts, int count, int max_n, int in_role, int out_role, int flags,
                       cudaStream_t st, int tail) {
    if (count == 1) {   // a CTA per row (column)
        const int nb = max_n > 8192 ? 8192 : max_n;
        LQ_LAUNCH(lq_pdl(k_prec_lower<4>, dim3(nb, count), kPrecThreads, 0, st, d_insts, in_role, flags));
        LQ_LAUNCH(lq_pdl(k_prec_upper<4>, dim3(nb, count), kPrecThreads, 0, st, d_insts, out_role, flags, tail));
    } else {            // a warp per row (column)
        int nb = (max_n + 3) / 4;
        nb = per_instance_blocks(nb > 8192 ? 8192 : nb, count);
        LQ_LAUNCH(lq_pdl(k_prec_lower<1>, dim3(nb, count), kPrecThreads, 0, st, d_insts, in_role, flags));
        LQ_LAUNCH(lq_pdl(k_prec_upper<1>, dim3(nb, count), kPrecThreads, 0, st, d_insts, out_role, flags, tail));
    }
}

void launch_chol_solve(const Inst* d_insts, int count, int max_n, int fp64, int in_role,
                       int out_role, int flags, cudaStream_t st) {
    size_t smem = 2 * (size_t)((max_n + kNb - 1) / kNb) * kNb * (fp64 ? 8 : 4);
    if (fp64) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_chol_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(lq_pdl(k_chol_solve<double>, dim3(1, count), solve_threads<double>(), smem, st, d_insts, in_role, out_role, flags));
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_chol_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(lq_pdl(k_chol_solve<float>, dim3(1, count), solve_threads<float>(), smem, st, d_insts, in_role, out_role, flags));
    }
}

}  // namespace lqmpc
