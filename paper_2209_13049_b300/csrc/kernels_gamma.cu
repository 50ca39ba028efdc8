// State elimination and products with the condensed Jacobian (Section II).
//
// Gamma (ns*N x nu*N) has block (r, t) = A^{r-t} B for t <= r (state x_{r+1},
// input u_t) and zero above.  The paper's conclusions note that all of its
// data sits in its first nu columns; the build stores only the G-stack
//   G[:, (N-1-k)*nu + c] = (A^k B)[:, c],   column-major, leading dim ldg,
// i.e. in reversed block order, so that row block r of Gamma is the
// contiguous column window G[:, (N-1-r)*nu : (N-1-r)*nu + n] with every column
// index >= n reading as zero.  The tensor-core SYRK exploits the same window
// through TMA coordinates.
#include "common.cuh"
#include "kernels.h"
#include "gamma_ff.cuh"

#include <algorithm>

namespace lqmpc {

// G_0 = B into its column block (N-1)*nu.
__global__ void k_gstack_init(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    const int total = I.ns * I.nu;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int i = q % I.ns, c = q / I.ns;
        I.G64[(size_t)I.ldg * ((I.N - 1) * I.nu + c) + i] = I.B[(size_t)c * I.ns + i];
    }
}

// G_k = A G_{k-1} (CSR A).  One thread per (row i, input c).
__global__ void k_gstack_step(const Inst* __restrict__ insts, int k) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (k >= I.N) return;
    const int total = I.ns * I.nu;
    const double* src = I.G64 + (size_t)I.ldg * ((I.N - k) * I.nu);
    double* dst = I.G64 + (size_t)I.ldg * ((I.N - 1 - k) * I.nu);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        int i = q % I.ns, c = q / I.ns;
        const double* sc = src + (size_t)I.ldg * c;
        double acc = 0.0;
        for (int p = I.a_ptr[i]; p < I.a_ptr[i + 1]; ++p) acc += I.a_val[p] * sc[I.a_idx[p]];
        dst[(size_t)I.ldg * c + i] = acc;
    }
}

// Working copies of the G-stack in FP32 and BF16 (padding rows stay zero).
__global__ void k_gstack_cast(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    const size_t total = (size_t)I.ldg * I.n;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        double g = I.G64[q];
        float gh = (float)g;
        if (I.G32) I.G32[q] = gh;
        if (I.G32lo) I.G32lo[q] = (float)(g - (double)gh);
        if (I.G16) I.G16[q] = __double2bfloat16(g);
        if (I.Gt) {
            unsigned t;   // round to the nearest TF32 (the tensor cores read 19 of the 32 bits)
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(gh));
            const float th = __uint_as_float(t);
            I.Gt[q] = th;
            I.Gtlo[q] = (float)(g - (double)th);
        }
    }
}

// out[r*ns + i] = sum_{t < (r+1) nu} G[i, (N-1-r) nu + t] v[t]   (out = Gamma v).
// Each lane owns one state i and RB consecutive row blocks; a G element
// loaded once serves every row block of the group (each is the same column
// window shifted by nu).  The KS warps of a CTA take consecutive slices of
// the column range and their partial sums are added in warp order
// (deterministic): an FP64 multiply-add holds one sub-partition's FP64 pipe
// for ~60 cycles on this part, so one warp per 32 states left most of each
// SM's four FP64 pipes idle behind a 500-long dependent chain.
template <int RB, int KS>
__global__ void __launch_bounds__(32 * KS) k_gamma_mv(const Inst* __restrict__ insts, int in_role, int out_role,
                                                      int flags) {
    pdl_wait();
    __shared__ double red[KS][RB][32];
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const double* v = role_ptr(I, in_role);
    double* out = role_ptr(I, out_role);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.z * RB;
    if (r0 >= I.N) return;
    const bool valid = i < I.ns;
    const int nu = I.nu, N = I.N, n = I.n;
    const int rlast = min(r0 + RB, N) - 1;
    double acc[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) acc[q] = 0.0;
    const int col0 = (N - 1 - rlast) * nu;       // smallest window start in the group
    const int c_beg = col0 + (n - col0) * w / KS, c_end = col0 + (n - col0) * (w + 1) / KS;
    const double* g = I.G64 + (valid ? i : 0);
    if (valid) {
        for (int col = c_beg; col < c_end; ++col) {
            const double gv = g[(size_t)I.ldg * col];
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                const int r = r0 + q;
                const int t = col - (N - 1 - r) * nu;
                if (r <= rlast && t >= 0) acc[q] += gv * __ldg(v + t);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q) red[w][q][lane] = acc[q];
    __syncthreads();
    if (w == 0 && valid) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            double s = red[0][q][lane];
#pragma unroll
            for (int k = 1; k < KS; ++k) s += red[k][q][lane];
            if (r0 + q <= rlast) out[(size_t)(r0 + q) * I.ns + i] = s;
        }
    }
}

// Gamma' w, two-level.  Stage 1: block (t, chunk, rgroup) computes, for input
// block t, a chunk of kTmvChunk states and kTmvRg consecutive row blocks
// r >= t of Gamma, the partial sums
//     P[rgroup][chunk][t*nu + c] = sum_{r in group} sum_{i in chunk} G[i, (N-1-r+t) nu + c] w_r[i]
// for NV vectors at once.  Stage 2 adds the partials in a fixed order
// (deterministic).  Small blocks over all three indices keep every SM busy:
// FP64 throughput per SM is low on this part, so the work must be spread.
constexpr int kTmvChunk = 128;
constexpr int kTmvRg = 8;
constexpr int kTmvMaxNu = 16;

__host__ __device__ inline int tmv_groups(int N) { return (N + kTmvRg - 1) / kTmvRg; }

template <int NV>
__global__ void __launch_bounds__(kTmvChunk) k_gamma_tmv_part(const Inst* __restrict__ insts, int w0_role,
                                                              int w1_role, int scale0, int flags) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int nchunks = (I.ns + kTmvChunk - 1) / kTmvChunk;
    const int ngroups = tmv_groups(I.N);
    const int t = blockIdx.x / ngroups, g = blockIdx.x % ngroups;
    const int chunk = blockIdx.z;
    if (t >= I.N || chunk >= nchunks) return;
    const int nu = I.nu, N = I.N;
    const int r0 = t + g * kTmvRg;
    double* part = I.gpart + ((size_t)g * nchunks + chunk) * NV * I.n;
    __shared__ double red[NV][kTmvMaxNu][kTmvChunk / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (r0 >= N) {   // empty group: contributes zeros
        for (int q = threadIdx.x; q < NV * nu; q += blockDim.x)
            part[(size_t)(q / nu) * I.n + t * nu + q % nu] = 0.0;
        return;
    }
    const int r1 = min(r0 + kTmvRg, N);
    const double* w0 = role_ptr(I, w0_role);
    const double* w1 = NV > 1 ? role_ptr(I, w1_role) : nullptr;
    const int i = chunk * kTmvChunk + threadIdx.x;
    for (int c0 = 0; c0 < nu; c0 += kTmvMaxNu) {
        const int cn = min(kTmvMaxNu, nu - c0);
        double acc[NV][kTmvMaxNu];
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
            for (int c = 0; c < kTmvMaxNu; ++c) acc[a][c] = 0.0;
        if (i < I.ns) {
            for (int r = r0; r < r1; ++r) {
                double wa = w0[(size_t)r * I.ns + i];
                if (scale0) wa *= I.sigx[(size_t)r * I.ns + i];
                double wb = NV > 1 ? w1[(size_t)r * I.ns + i] : 0.0;
                const double* gp = I.G64 + (size_t)I.ldg * ((N - 1 - r + t) * nu + c0) + i;
#pragma unroll
                for (int c = 0; c < kTmvMaxNu; ++c) {
                    if (c < cn) {
                        double gv = gp[(size_t)I.ldg * c];
                        acc[0][c] += gv * wa;
                        if (NV > 1) acc[NV - 1][c] += gv * wb;
                    }
                }
            }
        }
#pragma unroll
        for (int a = 0; a < NV; ++a)
#pragma unroll
            for (int c = 0; c < kTmvMaxNu; ++c) {
                if (c < cn) {
                    double v = warp_sum(acc[a][c]);
                    if (lane == 0) red[a][c][warp] = v;
                }
            }
        __syncthreads();
        const int nw = blockDim.x >> 5;
        for (int q = threadIdx.x; q < NV * cn; q += blockDim.x) {
            int a = q / cn, c = q % cn;
            double sum = 0.0;
            for (int w = 0; w < nw; ++w) sum += red[a][c][w];
            part[(size_t)a * I.n + t * nu + c0 + c] = sum;
        }
        __syncthreads();
    }
}

template <int NV>
__global__ void k_gamma_tmv_sum(const Inst* __restrict__ insts, int o0_role, int o1_role, int flags) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int nchunks = (I.ns + kTmvChunk - 1) / kTmvChunk;
    const int ngroups = tmv_groups(I.N);
    const double* part = I.gpart;
    double* o0 = role_ptr(I, o0_role);
    double* o1 = NV > 1 ? role_ptr(I, o1_role) : nullptr;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < I.n; j += gridDim.x * blockDim.x) {
        const int t = j / I.nu;
        const int gmax = tmv_groups(I.N - t);    // groups that hold row blocks of this t
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            double sum = 0.0;
            for (int g = 0; g < gmax && g < ngroups; ++g)
                for (int q = 0; q < nchunks; ++q)
                    sum += part[(((size_t)g * nchunks + q) * NV + a) * I.n + j];
            (a == 0 ? o0 : o1)[j] = sum;
        }
    }
}

// ---------------------------------------------------------------------------
// Float-float products (mixed-precision solves).  The G-stack is held as two
// FP32 planes (G32 + G32lo = G to ~48 bits) and each input as hi + lo; the
// products run on the FP32 pipes with error-free transformations (product
// error by FMA, sum error by TwoSum), about 2^-44 relative per term instead
// of FP64's 2^-53, at several times FP64's throughput on this part.
//
// Both products are small GEMMs with a block-triangular zero pattern:
//   Gamma v :   Y[i, r]   = sum_col G[i, col] V[col, r],   V[col, r] = v[col - off_r] (col >= off_r)
//   Gamma' w:   P[col, r] = sum_i   G[i, col] w_r[i],      needed where col >= off_r,
//               out[t nu + c] = sum_{d} P[(N-1-d) nu + c, t + d]
// with off_r = (N-1-r) nu.  Tiles entirely in the zero pattern are skipped;
// split-K partials are reduced in a fixed order.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void ff_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = sh + p;
    const float z = s - sh;
    const float t = (sh - (s - z)) + (p - z);
    sh = s;
    sl += t + e;
}


constexpr int kFfBM = 64, kFfBN = 16, kFfBK = 32, kFfThreads = 128;
constexpr int kFfLdT = kFfBK + 4;   // row stride of the transposed-product G tile (16-byte rows)

// 16-byte asynchronous global -> shared copy (zero-filled when !valid).
__device__ __forceinline__ void cp16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
// 4-byte asynchronous copy (zero-filled when !valid; src must then still be
// a valid address, it is not read).
__device__ __forceinline__ void cp4(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Split plan of Gamma v: r-tile t holds rows N - 16 (t + 1) .. N - 16 t - 1
// (aligned to the horizon's end), needs the columns from kbeg on (nk K-tiles
// of 32) and gives them to S = min(nk, kFfMaxSplits) CTAs, so that every CTA
// of the launch gets one K-tile (two past 512 columns) whatever its r-tile.
__host__ __device__ inline void mv_ff_rtile(int t, int N, int nu, int n, int& kbeg, int& nk, int& S,
                                            int cap = kFfMaxSplits) {
    const int r1 = N - kFfBN * t;
    kbeg = ((N - r1) * nu) / kFfBK * kFfBK;
    nk = (n - kbeg + kFfBK - 1) / kFfBK;
    S = nk < cap ? nk : cap;
}

// Gamma v: block (r-tile, m-tile of states, split of the column range).  G
// tiles stream through a double-buffered shared-memory ring (cp.async); the
// input comes split into float-float (by k_ff_prep_v, or by the kernel that
// formed it: kFuseInSplit).  Each block leaves its
// split's partial tile.  With kFuseSumHere (batches) the last of the tile's
// splits to arrive (a counter per tile, acquire-release like last_arrival)
// sums them in split order, as k_gamma_mv_ff_sum does for one instance, and
// writes the output with its fused uses (kFuseOutW, kFuseOutDxs).  For one
// instance few CTAs arrive last, each summing eight outputs in turn, which
// took longer than the separate sum launch it saves (C2: 15.7 -> 17.3 ms);
// a batch has many more tiles (256 instances: 845 -> 833 ms).
__global__ void __launch_bounds__(kFfThreads) k_gamma_mv_ff(const Inst* __restrict__ insts, int in_role,
                                                            int out_role, int flags, int fuse, int cap) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int ns = I.ns, nu = I.nu, N = I.N, n = I.n, ldg = I.ldg;
    const int mt = (ns + kFfBM - 1) / kFfBM, nt = (N + kFfBN - 1) / kFfBN;
    // r tiles aligned to the horizon's end (rows r0 .. r1-1, r0 may be
    // negative): the partial tile holds the first stages, which need only the
    // last columns (col >= off_{r1-1})
    int rem = blockIdx.x, t = 0, kbeg = 0, nk = 0, S = 1;
    for (;; ++t) {
        if (t >= nt) return;
        mv_ff_rtile(t, N, nu, n, kbeg, nk, S, cap);
        if (rem < mt * S) break;
        rem -= mt * S;
    }
    const int split = rem % S;
    const int m0 = (rem / S) * kFfBM, r1 = N - kFfBN * t, r0 = r1 - kFfBN;
    const double* v = role_ptr(I, in_role);
    const int k0t = nk * split / S, k1t = nk * (split + 1) / S;
    __shared__ __align__(16) float Gs[2][2][kFfBK][kFfBM];          // [buffer][hi, lo][col][state]
    __shared__ float Vs[2][2][kFfBK][kFfBN + 1];                   // [buffer][hi, lo][col][r]
    (void)v;
    const float* vsp = I.ffv;                                       // the input, split into float-float
    auto load = [&](int kt, int buf) {
        const int c0 = kbeg + kt * kFfBK;
        for (int e = threadIdx.x; e < kFfBK * (kFfBM / 4); e += kFfThreads) {
            const int kk = e / (kFfBM / 4), q = e % (kFfBM / 4);
            const int col = c0 + kk;
            const bool ok = col < n;
            const size_t off = (size_t)ldg * (ok ? col : 0) + m0 + 4 * q;   // rows past ns are zero padding
            cp16(&Gs[buf][0][kk][4 * q], I.G32 + off, ok);
            cp16(&Gs[buf][1][kk][4 * q], I.G32lo + off, ok);
        }
        // the Toeplitz-gathered input tile, asynchronous like the G tiles
        for (int e = threadIdx.x; e < kFfBK * kFfBN; e += kFfThreads) {
            const int kk = e / kFfBN, rr = e % kFfBN;
            const int col = c0 + kk, r = r0 + rr;
            const int t = (col < n && r >= 0) ? col - (N - 1 - r) * nu : -1;
            const bool ok = t >= 0;
            cp4(&Vs[buf][0][kk][rr], vsp + (ok ? t : 0), ok);
            cp4(&Vs[buf][1][kk][rr], vsp + n + (ok ? t : 0), ok);
        }
        cp_commit();
    };
    const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;   // 8 x 16 threads: 2 r x 4 states each
    float sh[4][2], sl[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) sh[a][b] = sl[a][b] = 0.f;
    if (k0t < k1t) load(k0t, 0);
    for (int kt = k0t; kt < k1t; ++kt) {
        const int buf = (kt - k0t) & 1;
        if (kt + 1 < k1t) {
            load(kt + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kFfBK; ++kk) {
            float ah[4], al[4], bh[2], bl[2];
#pragma unroll
            for (int a = 0; a < 4; ++a) { ah[a] = Gs[buf][0][kk][ty + 16 * a]; al[a] = Gs[buf][1][kk][ty + 16 * a]; }
#pragma unroll
            for (int b = 0; b < 2; ++b) { bh[b] = Vs[buf][0][kk][tx + 8 * b]; bl[b] = Vs[buf][1][kk][tx + 8 * b]; }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) ff_mac(sh[a][b], sl[a][b], ah[a], al[a], bh[b], bl[b]);
        }
        __syncthreads();
    }
    // the output and its fused uses from a tile's float-float sum
    auto emit = [&](size_t k, float hs, float ls) {
        const double sum = (double)hs + (double)ls;
        role_ptr(I, out_role)[k] = sum;
        if (fuse & kFuseOutDxs) I.dxs[k] = sum;
        if (fuse & kFuseOutW) {
            float h, l;
            split_ff(sum * I.sigx[k], h, l);
            I.ffw[k] = h;
            I.ffw[(size_t)I.SX + k] = l;
        }
    };
    if ((fuse & kFuseSumHere) && S == 1) {   // the tile's only split: no partial, no count
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int i = m0 + ty + 16 * a, r = r0 + tx + 8 * b;
                if (i >= ns || r < 0) continue;
                float hs = 0.f, ls = 0.f;
                ff_acc(hs, ls, sh[a][b], sl[a][b]);
                emit((size_t)r * ns + i, hs, ls);
            }
        return;
    }
    // partial[split][r][i], float-float
    float2* part = ff_parts(I) + (size_t)split * I.SX;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = m0 + ty + 16 * a, r = r0 + tx + 8 * b;
            if (i < ns && r >= 0) part[(size_t)r * ns + i] = make_float2(sh[a][b], sl[a][b]);
        }
    if (!(fuse & kFuseSumHere)) return;
    __shared__ int last_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int* cnt = I.mvcnt + (size_t)t * mt + m0 / kFfBM;
        int old;
        asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], 1;" : "=r"(old) : "l"(cnt) : "memory");
        last_sh = old == S - 1;
        if (last_sh) atomicExch(cnt, 0);
    }
    __syncthreads();
    if (!last_sh) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = m0 + ty + 16 * a, r = r0 + tx + 8 * b;
            if (i >= ns || r < 0) continue;
            const size_t k = (size_t)r * ns + i;
            float2 pv[kFfMaxSplits];   // every split's partial in flight at once, summed in split order
#pragma unroll
            for (int q = 0; q < kFfMaxSplits; ++q)
                pv[q] = q < S ? __ldcg(ff_parts(I) + (size_t)q * I.SX + k) : make_float2(0.f, 0.f);
            float hs = 0.f, ls = 0.f;
#pragma unroll
            for (int q = 0; q < kFfMaxSplits; ++q) ff_acc(hs, ls, pv[q].x, pv[q].y);
            emit(k, hs, ls);
        }
}

// out = sum of the split partials; with kFuseOutW also the float-float split
// of Sigma_x out (the operand of a following Gamma' (Sigma_x .)), with
// kFuseOutDxs also a copy into dxs.
__global__ void k_gamma_mv_ff_sum(const Inst* __restrict__ insts, int out_role, int flags, int splits, int fuse) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    double* out = role_ptr(I, out_role);
    (void)splits;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < I.SX; k += gridDim.x * blockDim.x) {
        // the splits of row r's r-tile (the split plan of k_gamma_mv_ff)
        int kbeg, nk, S;
        mv_ff_rtile((I.N - 1 - k / I.ns) / kFfBN, I.N, I.nu, I.n, kbeg, nk, S);
        float2 pv[kFfMaxSplits];   // every split's partial in flight at once, summed in split order
#pragma unroll
        for (int q = 0; q < kFfMaxSplits; ++q)
            pv[q] = q < S ? ff_parts(I)[(size_t)q * I.SX + k] : make_float2(0.f, 0.f);
        float hs = 0.f, ls = 0.f;
#pragma unroll
        for (int q = 0; q < kFfMaxSplits; ++q) ff_acc(hs, ls, pv[q].x, pv[q].y);
        const double s = (double)hs + (double)ls;
        out[k] = s;
        if (fuse & kFuseOutDxs) I.dxs[k] = s;
        if (fuse & kFuseOutW) {
            float h, l;
            split_ff(s * I.sigx[k], h, l);
            I.ffw[k] = h;
            I.ffw[(size_t)I.SX + k] = l;
        }
    }
}

// Float-float split of the Gamma operand, once per product.
__global__ void k_ff_prep_v(const Inst* __restrict__ insts, int in_role, int flags) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const double* v = role_ptr(I, in_role);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < I.n; j += gridDim.x * blockDim.x)
        split_ff(v[j], I.ffv[j], I.ffv[I.n + j]);
}

// Float-float split of the Gamma' operands (w0 scaled by Sigma_x when
// scale0), once per product instead of once per tile that reads them.
__global__ void k_ff_prep_w(const Inst* __restrict__ insts, int w0_role, int w1_role, int scale0, int flags) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const double* w0 = role_ptr(I, w0_role);
    const double* w1 = w1_role != R_NONE ? role_ptr(I, w1_role) : nullptr;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < I.SX; k += gridDim.x * blockDim.x) {
        float h, l;
        double wv = w0[k];
        if (scale0) wv *= I.sigx[k];
        split_ff(wv, h, l);
        I.ffw[k] = h;
        I.ffw[(size_t)I.SX + k] = l;
        if (w1) {
            split_ff(w1[k], h, l);
            I.ffw[2 * (size_t)I.SX + k] = h;
            I.ffw[3 * (size_t)I.SX + k] = l;
        }
    }
}

// Gamma' w for NV vectors: P[col, r'] over r' = vec * N + r, K = states.  G
// tiles (transposed: [col][state]) and the pre-split operands stream through
// a double-buffered ring.
template <int NV>
__global__ void __launch_bounds__(kFfThreads) k_gamma_tmv_ff(const Inst* __restrict__ insts, int w0_role,
                                                             int w1_role, int scale0, int flags, int splits) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int ns = I.ns, nu = I.nu, N = I.N, n = I.n, ldg = I.ldg;
    const int NR = NV * N;
    // r tiles per vector aligned to the horizon's end: the partial tile holds
    // the first stages, whose useful columns are only the last few blocks
    const int tpv = (N + kFfBN - 1) / kFfBN;
    const int mt = (n + kFfBM - 1) / kFfBM, nt = NV * tpv;
    const int tile = blockIdx.x / splits, split = blockIdx.x % splits;
    if (tile >= mt * nt) return;
    const int rt = tile / mt, vec_t = rt / tpv;
    const int c0 = (tile % mt) * kFfBM, r_lo = N - kFfBN * (rt % tpv + 1);   // rows r_lo .. r_lo + 15 (r >= 0)
    // skip tiles wholly in the unused triangle: need some col >= off_r
    {
        bool any = false;
        for (int r = max(r_lo, 0); r < r_lo + kFfBN && !any; ++r)
            if (min(c0 + kFfBM, n) - 1 >= (N - 1 - r) * nu) any = true;
        if (!any) return;
    }
    (void)w0_role; (void)w1_role; (void)scale0;   // operands come split by k_ff_prep_w
    const int nk = (ns + kFfBK - 1) / kFfBK;
    const int k0t = nk * split / splits, k1t = nk * (split + 1) / splits;
    __shared__ __align__(16) float Gs[2][2][kFfBM][kFfLdT];   // [buffer][hi, lo][col][state]
    __shared__ float Ws[2][2][kFfBK][kFfBN + 1];              // [buffer][hi, lo][state][r']
    auto load = [&](int kt, int buf) {
        const int i0 = kt * kFfBK;
        for (int e = threadIdx.x; e < kFfBM * (kFfBK / 4); e += kFfThreads) {
            const int mm = e / (kFfBK / 4), q = e % (kFfBK / 4);
            const int col = c0 + mm;
            const bool ok = col < n;                  // states past ns are zero padding
            const size_t off = (size_t)ldg * (ok ? col : 0) + i0 + 4 * q;
            cp16(&Gs[buf][0][mm][4 * q], I.G32 + off, ok);
            cp16(&Gs[buf][1][mm][4 * q], I.G32lo + off, ok);
        }
        for (int e = threadIdx.x; e < kFfBK * kFfBN; e += kFfThreads) {
            const int rr = e / kFfBK, kk = e % kFfBK;
            const int r = r_lo + rr, i = i0 + kk;
            const bool ok = r >= 0 && i < ns;
            const size_t q = ok ? (size_t)r * ns + i : 0;
            cp4(&Ws[buf][0][kk][rr], I.ffw + (size_t)(2 * vec_t) * I.SX + q, ok);
            cp4(&Ws[buf][1][kk][rr], I.ffw + (size_t)(2 * vec_t + 1) * I.SX + q, ok);
        }
        cp_commit();
    };
    const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;
    float sh[4][2], sl[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) sh[a][b] = sl[a][b] = 0.f;
    if (k0t < k1t) load(k0t, 0);
    for (int kt = k0t; kt < k1t; ++kt) {
        const int buf = (kt - k0t) & 1;
        if (kt + 1 < k1t) {
            load(kt + 1, buf ^ 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kFfBK; ++kk) {
            float ah[4], al[4], bh[2], bl[2];
#pragma unroll
            for (int a = 0; a < 4; ++a) { ah[a] = Gs[buf][0][ty + 16 * a][kk]; al[a] = Gs[buf][1][ty + 16 * a][kk]; }
#pragma unroll
            for (int b = 0; b < 2; ++b) { bh[b] = Ws[buf][0][kk][tx + 8 * b]; bl[b] = Ws[buf][1][kk][tx + 8 * b]; }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) ff_mac(sh[a][b], sl[a][b], ah[a], al[a], bh[b], bl[b]);
        }
        __syncthreads();
    }
    // partial[split] skewed along the anti-diagonals Gamma' sums: P[col, r']
    // with col = (N-1-d) nu + c and r' = vec N + r goes to [vec][t][c][d],
    // t = r - d, so the terms of one output are contiguous; t < 0 is not used
    float2* part = ff_parts(I) + (size_t)split * NR * n;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int col = c0 + ty + 16 * a, r = r_lo + tx + 8 * b;
            if (col < n && r >= 0) {
                const int d = N - 1 - col / nu, c = col % nu, t = r - d;
                if (t >= 0) part[(((size_t)vec_t * N + t) * nu + c) * N + d] = make_float2(sh[a][b], sl[a][b]);
            }
        }
}

// Gamma' w from the split partials: one warp per output.  With rhs (one
// vector, the corrector's Gamma' w) the warp also writes the right-hand side
// b = -r_d + Gamma' w + w_u of that output.
template <int NV>
__global__ void k_gamma_tmv_ff_sum(const Inst* __restrict__ insts, int o0_role, int o1_role, int flags,
                                   int splits, int rhs) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int n = I.n, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int q = blockIdx.x * wpb + (threadIdx.x >> 5); q < NV * n; q += gridDim.x * wpb) {
        const int vec = q / n, j = q % n;
        const double s = gamma_tmv_ff_gather(I, NV, vec, j, splits);
        if (lane == 0) {
            (vec == 0 ? role_ptr(I, o0_role) : role_ptr(I, o1_role))[j] = s;
            if (NV == 1 && rhs) I.b[j] = -I.rd[j] + s + I.wxu[j];
        }
    }
}

// Free response y_t = A y_{t-1} + w_{t-1} for t = 1..N, y_0 = xbar (w = 0
// when absent; one block per instance, sequential in t).
__global__ void k_ychain(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    const double* prev = I.xbar;
    for (int t = 0; t < I.N; ++t) {
        double* cur = I.y + (size_t)t * I.ns;
        for (int i = threadIdx.x; i < I.ns; i += blockDim.x) {
            double acc = 0.0;
            for (int p = I.a_ptr[i]; p < I.a_ptr[i + 1]; ++p) acc += I.a_val[p] * prev[I.a_idx[p]];
            if (I.wd) acc += I.wd[(size_t)t * I.ns + i];
            cur[i] = acc;
        }
        __syncthreads();
        prev = cur;
    }
}

// w = Qbar y (Q on blocks 0..N-2, Qf on block N-1), CSR, into tmpx.
__global__ void k_qbar_y(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < I.SX; k += gridDim.x * blockDim.x) {
        int r = k / I.ns, i = k % I.ns;
        bool last = r == I.N - 1;
        const int* ptr = last ? I.qf_ptr : I.q_ptr;
        const int* idx = last ? I.qf_idx : I.q_idx;
        const double* val = last ? I.qf_val : I.q_val;
        const double* yr = I.y + (size_t)r * I.ns;
        double acc = 0.0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) acc += val[p] * yr[idx[p]];
        I.tmpx[k] = acc;
    }
}

// Dense-Q operand for H: GQ = Q * G (columns of the G-stack), or Qf * G.
__global__ void k_q_times_g(const Inst* __restrict__ insts, int use_qf, double* out) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    const int* ptr = use_qf ? I.qf_ptr : I.q_ptr;
    const int* idx = use_qf ? I.qf_idx : I.q_idx;
    const double* val = use_qf ? I.qf_val : I.q_val;
    const size_t total = (size_t)I.ns * I.n;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(q % I.ns);
        size_t col = q / I.ns;
        const double* g = I.G64 + (size_t)I.ldg * col;
        double acc = 0.0;
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) acc += val[p] * g[idx[p]];
        out[(size_t)I.ldg * col + i] = acc;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

void launch_gstack(const Inst* d_inst, const Inst& h, cudaStream_t st) {
    int tot = h.ns * h.nu;
    int nb = (tot + 255) / 256;
    nb = nb > 4096 ? 4096 : nb;
    LQ_LAUNCH(lq_pdl(k_gstack_init, dim3(nb, 1), 256, 0, st, d_inst));
    LQ_LAUNCH(for (int k = 1; k < h.N; ++k) lq_pdl(k_gstack_step, dim3(nb, 1), 256, 0, st, d_inst, k));
    size_t tot2 = (size_t)h.ldg * h.n;
    int nb2 = (int)((tot2 + 255) / 256);
    nb2 = nb2 > 8192 ? 8192 : nb2;
    LQ_LAUNCH(lq_pdl(k_gstack_cast, dim3(nb2, 1), 256, 0, st, d_inst));
}

void launch_gamma_mv(const Inst* d_insts, int count, int max_ns, int max_N, int in_role,
                     int out_role, int flags, cudaStream_t st) {
    constexpr int RB = 4, KS = 8;
    dim3 grid((max_ns + 31) / 32, count, (max_N + RB - 1) / RB);
    LQ_LAUNCH(lq_pdl(k_gamma_mv<RB, KS>, grid, 32 * KS, 0, st, d_insts, in_role, out_role, flags));
}

size_t gamma_tmv_part_doubles(int ns, int n, int N) {
    size_t fp64 = (size_t)2 * tmv_groups(N) * ((ns + kTmvChunk - 1) / kTmvChunk) * n;
    size_t ff_mv = (size_t)kFfMaxSplits * ns * N;
    size_t ff_tmv = (size_t)kFfMaxSplits * 2 * N * n;
    return std::max(fp64, std::max(ff_mv, ff_tmv));
}

void launch_gamma_tmv(const Inst* d_insts, int count, int max_ns, int max_N, int max_n,
                      int w0_role, int w1_role, int o0_role, int o1_role, int scale0, int flags,
                      cudaStream_t st) {
    int nchunks = (max_ns + kTmvChunk - 1) / kTmvChunk;
    dim3 grid(max_N * tmv_groups(max_N), count, nchunks);
    int nbs = (max_n + 255) / 256;
    if (w1_role != R_NONE) {
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_part<2>, grid, kTmvChunk, 0, st, d_insts, w0_role, w1_role, scale0, flags));
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_sum<2>, dim3(nbs, count), 256, 0, st, d_insts, o0_role, o1_role, flags));
    } else {
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_part<1>, grid, kTmvChunk, 0, st, d_insts, w0_role, R_NONE, scale0, flags));
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_sum<1>, dim3(nbs, count), 256, 0, st, d_insts, o0_role, R_NONE, flags));
    }
}

// A CTA's K range is kept to kFfMaxKt K-tiles at most: in a batch the SMs are
// full of tiles anyway, and the largest instances' CTAs would otherwise run
// the whole range (63 K-tiles at ns = 2000) well after the rest.  256-instance
// batch: 688 ms unbounded, 657 / 643 / 677 ms with 32 / 16 / 8.
constexpr int kFfMaxKt = 16;

static int ff_splits(int tiles, int nk) {
    int s = (4 * device_sm_count() + tiles - 1) / (tiles > 0 ? tiles : 1);   // about four CTAs per SM
    if (s > nk) s = nk;
    if (s > kFfMaxSplits) s = kFfMaxSplits;
    return s < 1 ? 1 : s;
}

void launch_gamma_mv_ff(const Inst* d_insts, int count, int max_ns, int max_N, int max_n, int in_role,
                        int out_role, int flags, cudaStream_t st, int fuse) {
    // CTAs: sum over r-tiles of m-tiles x splits (exact for one instance; for
    // a batch a bound over its instances, the surplus CTAs return at once).
    // One instance splits K up to kFfMaxSplits ways to fill the SMs; a batch
    // has tiles enough across its instances, so its split count is capped at
    // what makes about four CTAs per SM (one at 256 instances: 16-way splits
    // had launched half a million CTAs, nearly all returning at once).
    const int mt = (max_ns + kFfBM - 1) / kFfBM, nt = (max_N + kFfBN - 1) / kFfBN;
    int ctas = 0, cap = kFfMaxSplits;
    if (count == 1) {
        for (int t = 0; t < nt; ++t) {
            int kbeg, nk, S;
            mv_ff_rtile(t, max_N, max_n / max_N, max_n, kbeg, nk, S);
            ctas += mt * S;
        }
    } else {
        const long long tiles = (long long)count * mt * nt;
        const long long want = 4LL * device_sm_count();
        cap = (int)((want + tiles - 1) / tiles);
        const int nkmax = (max_n + kFfBK - 1) / kFfBK, cap_len = (nkmax + kFfMaxKt - 1) / kFfMaxKt;
        cap = cap > cap_len ? cap : cap_len;
        cap = cap < 1 ? 1 : (cap > kFfMaxSplits ? kFfMaxSplits : cap);
        ctas = mt * nt * (nkmax < cap ? nkmax : cap);
    }
    if (!(fuse & kFuseInSplit))
        LQ_LAUNCH(lq_pdl(k_ff_prep_v, dim3((max_n + 255) / 256, count), 256, 0, st, d_insts, in_role, flags));
    if (count > 1) {   // the split-K sum by the last split of each tile
        LQ_LAUNCH(lq_pdl(k_gamma_mv_ff, dim3(ctas, count), kFfThreads, 0, st, d_insts, in_role, out_role, flags,
                         fuse | kFuseSumHere, cap));
    } else {
        LQ_LAUNCH(lq_pdl(k_gamma_mv_ff, dim3(ctas, count), kFfThreads, 0, st, d_insts, in_role, out_role, flags, fuse,
                         cap));
        const int nb = (max_ns * max_N + 255) / 256;
        LQ_LAUNCH(lq_pdl(k_gamma_mv_ff_sum, dim3(nb > 4096 ? 4096 : nb, count), 256, 0, st, d_insts, out_role, flags,
                         0, fuse));
    }
}

int gamma_tmv_ff_splits(int count, int max_ns, int max_N, int max_n, int NV) {
    const int tiles = ((max_n + kFfBM - 1) / kFfBM) * (NV * ((max_N + kFfBN - 1) / kFfBN));
    const int nk = (max_ns + kFfBK - 1) / kFfBK;
    const int s = ff_splits(tiles * count / 2, nk), s_len = (nk + kFfMaxKt - 1) / kFfMaxKt;
    return s > s_len ? s : (s_len > kFfMaxSplits ? kFfMaxSplits : s_len);
}

void launch_gamma_tmv_ff(const Inst* d_insts, int count, int max_ns, int max_N, int max_n, int w0_role,
                         int w1_role, int o0_role, int o1_role, int scale0, int flags, cudaStream_t st, int fuse) {
    const int NV = w1_role != R_NONE ? 2 : 1;
    const int tiles = ((max_n + kFfBM - 1) / kFfBM) * (NV * ((max_N + kFfBN - 1) / kFfBN));
    const int splits = gamma_tmv_ff_splits(count, max_ns, max_N, max_n, NV);
    int nb = (NV * max_n + 1) / 2;   // two warps (two outputs) per CTA: every SM takes part
    nb = per_instance_blocks(nb > 8192 ? 8192 : nb, count);
    int npre = (max_ns * max_N + 255) / 256;
    npre = npre > 4096 ? 4096 : npre;
    if (!(fuse & kFuseInSplit))
        LQ_LAUNCH(lq_pdl(k_ff_prep_w, dim3(npre, count), 256, 0, st, d_insts, w0_role, w1_role, scale0, flags));
    if (NV == 2) {
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_ff<2>, dim3(tiles * splits, count), kFfThreads, 0, st, d_insts, w0_role, w1_role, scale0, flags, splits));
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_ff_sum<2>, dim3(nb, count), 64, 0, st, d_insts, o0_role, o1_role, flags, splits,
                         0));
    } else {
        LQ_LAUNCH(lq_pdl(k_gamma_tmv_ff<1>, dim3(tiles * splits, count), kFfThreads, 0, st, d_insts, w0_role, R_NONE, scale0, flags, splits));
        if (!(fuse & kFuseNoSum))
            LQ_LAUNCH(lq_pdl(k_gamma_tmv_ff_sum<1>, dim3(nb, count), 64, 0, st, d_insts, o0_role, R_NONE, flags, splits,
                             (fuse & kFuseRhs) ? 1 : 0));
    }
}

// The cross term x_t' S u_t of the stage cost in the condensed Hessian:
// H[j, l] += (G_{t-1-k}' S)[a, b] for input j = (k, a) of an earlier stage
// than input l = (t, b), and its mirror below the diagonal (one thread per
// entry, each computing its own dot product over the states).
__global__ void k_hess_cross(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (!I.Sx) return;
    const int n = I.n, nu = I.nu, N = I.N, ns = I.ns;
    const size_t total = (size_t)n * n;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q % n), l = (int)(q / n);
        const int kj = j / nu, kl = l / nu;
        if (kj == kl) continue;
        // earlier stage e with input index ae, later stage t with index bt
        const int e = kj < kl ? kj : kl, t = kj < kl ? kl : kj;
        const int ae = kj < kl ? j % nu : l % nu, bt = kj < kl ? l % nu : j % nu;
        const double* g = I.G64 + (size_t)I.ldg * ((N - 1 - (t - 1 - e)) * nu + ae);
        const double* sc = I.Sx + (size_t)bt * ns;
        double v = 0.0;
        for (int i = 0; i < ns; ++i) v += g[i] * sc[i];
        I.H64[q] += v;
    }
}

// h_t += S' y_t (y_0 = xbar): the cross term's part of the condensed linear
// term (one warp per output).
__global__ void k_h_cross(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (!I.Sx) return;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int q = blockIdx.x * wpb + (threadIdx.x >> 5); q < I.n; q += gridDim.x * wpb) {
        const int t = q / I.nu, b = q % I.nu;
        const double* yt = t == 0 ? I.xbar : I.y + (size_t)(t - 1) * I.ns;
        const double* sc = I.Sx + (size_t)b * I.ns;
        double v = 0.0;
        for (int i = lane; i < I.ns; i += 32) v += sc[i] * yt[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) I.h[q] += v;
    }
}

void launch_hess_cross(const Inst* d_inst, int n, cudaStream_t st) {
    size_t tot = (size_t)n * n;
    int nb = (int)((tot + 255) / 256);
    nb = nb > 8192 ? 8192 : nb;
    LQ_LAUNCH(lq_pdl(k_hess_cross, dim3(nb, 1), 256, 0, st, d_inst));
}

void launch_h_cross(const Inst* d_insts, int count, int max_n, cudaStream_t st) {
    int nb = (max_n + 7) / 8;
    nb = per_instance_blocks(nb > 4096 ? 4096 : nb, count);
    LQ_LAUNCH(lq_pdl(k_h_cross, dim3(nb, count), 256, 0, st, d_insts));
}

void launch_ychain(const Inst* d_insts, int count, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_ychain, dim3(1, count), 1024, 0, st, d_insts));
}

void launch_qbar_y(const Inst* d_insts, int count, int max_sx, cudaStream_t st) {
    int nb = (max_sx + 255) / 256;
    nb = nb > 4096 ? 4096 : nb;
    LQ_LAUNCH(lq_pdl(k_qbar_y, dim3(nb, count), 256, 0, st, d_insts));
}

void launch_q_times_g(const Inst* d_inst, const Inst& h, int use_qf, double* out, cudaStream_t st) {
    size_t tot = (size_t)h.ns * h.n;
    int nb = (int)((tot + 255) / 256);
    nb = nb > 8192 ? 8192 : nb;
    LQ_LAUNCH(lq_pdl(k_q_times_g, dim3(nb, 1), 256, 0, st, d_inst, use_qf, out));
}

}  // namespace lqmpc
