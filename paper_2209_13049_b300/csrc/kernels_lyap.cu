// FP64 condensed KKT matrix (Eq. 7) for plants whose A is sparse, without
// the SYRK: Horner chains over the horizon, one per block column.
//
// With Gamma's blocks G_d = A^d B (Section II), block (c1, c) of
// Gamma' Sigma_x Gamma for c1 <= c is
//     sum_{r >= c} (A^{r-c1} B)' Sigma_r A^{r-c} B = B' (A')^{c-c1} W_c,
//     W_c = sum_{d >= 0} (A')^d Sigma_{c+d} G_d.
// Column `col` of W_c comes from Horner's scheme backwards in d,
//     z <- Sigma_{N-1} G_{N-1-c}[:, col];  z <- A' z + Sigma_{c+d} G_d[:, col]  (d = N-2-c .. 0),
// and then z <- A' z walks c1 = c-1 .. 0, each z giving the entries
// B' z of column `col` of block (c1, c).  One CTA per (c, col): N sparse
// products A' z per CTA (2 nnz(A) flop each), no ns x ns intermediates and no
// dense products with the G-stack: N^2 nu nnz(A) + N(N+1)/2 nu (ns + nnz(B))
// multiply-adds, ~15x fewer FP64 operations than the SYRK and ~4x fewer than
// the recursion P_c = Sigma_c + A' P_{c+1} A with its block products G_d' W_c,
// for the 2-D heat plants (FP64 runs at 1/64 of the FP32 rate on this part).
// The same matrix up to rounding order.
//
// A' is available as CSR (the columns of A); B's nonzeros as per-column
// lists.  For batches blockIdx.x runs over the largest (N, nu) and CTAs
// outside an instance's own sizes return.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

__global__ void k_ly_chain(const Inst* __restrict__ insts, int flags, int max_nu, double shift) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int ns = I.ns, nu = I.nu, N = I.N, n = I.n, ldg = I.ldg;
    const int c = blockIdx.x / max_nu, col = blockIdx.x % max_nu;
    if (c >= N || col >= nu) return;
    extern __shared__ double zs[];
    double* z0 = zs;
    double* z1 = zs + ns;
    // z = A' z_old + Sigma_{c+d} G_d[:, col]  (scaled term only when d >= 0)
    auto step = [&](const double* zin, double* zout, int d) {
        const double* sg = d >= 0 ? I.sigx + (size_t)(c + d) * ns : nullptr;
        const double* g = d >= 0 ? I.G64 + (size_t)ldg * ((N - 1 - d) * nu + col) : nullptr;
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            double acc = sg ? sg[i] * g[i] : 0.0;
            for (int p = I.at_ptr[i]; p < I.at_ptr[i + 1]; ++p) acc += I.at_val[p] * zin[I.at_idx[p]];
            zout[i] = acc;
        }
        __syncthreads();
    };
    // W_c[:, col]
    {
        const int d = N - 1 - c;
        const double* sg = I.sigx + (size_t)(N - 1) * ns;
        const double* g = I.G64 + (size_t)ldg * ((N - 1 - d) * nu + col);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) z0[i] = sg[i] * g[i];
        __syncthreads();
    }
    for (int d = N - 2 - c; d >= 0; --d) {
        step(z0, z1, d);
        double* t = z0; z0 = z1; z1 = t;
    }
    // blocks (c1, c), c1 = c .. 0: entries B' z, one warp per row a of the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c1 = c; c1 >= 0; --c1) {
        if (c1 < c) {
            step(z0, z1, -1);
            double* t = z0; z0 = z1; z1 = t;
        }
        for (int a = warp; a < nu; a += nw) {
            double s = 0.0;
            for (int p = I.bc_ptr[a] + lane; p < I.bc_ptr[a + 1]; p += 32) s += I.bc_val[p] * z0[I.bc_idx[p]];
            s = warp_sum(s);
            if (lane == 0) {
                const int row = c1 * nu + a, cc = c * nu + col;
                double v = s + I.H64[(size_t)row + (size_t)n * cc];
                if (row == cc) v = (v + I.sigu[row]) * (1.0 + shift);   // shift: a retried factor
                // within the diagonal block each pair is computed twice (by
                // the CTAs of both columns): the lower one is written to both
                if (c1 < c || row >= cc) I.M64[(size_t)row + (size_t)n * cc] = v;
                if (c1 < c || row > cc) I.M64[(size_t)cc + (size_t)n * row] = v;
            }
        }
        // the next step overwrites the other buffer only; the dots above read
        // z0, which the step after it overwrites behind a barrier
    }
}

// The same chains in float-float on the FP32 pipes (FP64 runs at 1/64 of
// its rate here): z as hi + lo planes in shared memory, A', B and G (G32 +
// G32lo) as float-float pairs, Sigma_x split once per launch into sig_ff;
// every multiply-add is an exact FP32 product (FMA) plus the cross terms,
// summed by TwoSum.  About 2^-44 relative per operation, ~1e-12 after the
// horizon's 50 steps: M for the two-level FP32 tier, whose E = M - L1 L1'
// needs M far below FP32 rounding, not at FP64's.
namespace {
__device__ __forceinline__ void ffc_mac(float& ah, float& al, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    const float s = ah + p;
    const float z = s - ah;
    al += ((ah - (s - z)) + (p - z)) + e;
    ah = s;
}
}  // namespace

__global__ void k_sig_split(const Inst* __restrict__ insts, int flags) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int sx = I.SX;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < sx; k += gridDim.x * blockDim.x) {
        const double v = I.sigx[k];
        const float h = (float)v;
        I.sig_ff[k] = h;
        I.sig_ff[sx + k] = (float)(v - (double)h);
    }
}

__global__ void k_ly_chain_ff(const Inst* __restrict__ insts, int flags, int max_nu, double shift) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const int ns = I.ns, nu = I.nu, N = I.N, n = I.n, ldg = I.ldg, sx = I.SX;
    const int c = blockIdx.x / max_nu, col = blockIdx.x % max_nu;
    if (c >= N || col >= nu) return;
    extern __shared__ float2 zf2[];    // z as (hi, lo) pairs, two buffers
    float2* z0 = zf2;
    float2* z1 = zf2 + ns;
    // A' packed per nonzero as (column index, hi, lo): one 16-byte load each
    const int4* ap = reinterpret_cast<const int4*>(I.at_pack);
    // z <- A' z_old + Sigma_{c+d} G_d[:, col]  (scaled term only when d >= 0)
    auto step = [&](const float2* zin, float2* zout, int d) {
        const float* sh = I.sig_ff + (size_t)(c + (d >= 0 ? d : 0)) * ns;
        const float* sl = sh + sx;
        const size_t go = (size_t)ldg * ((N - 1 - (d >= 0 ? d : 0)) * nu + col);
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            float th = 0.f, tl = 0.f;
            if (d >= 0) ffc_mac(th, tl, sh[i], sl[i], I.G32[go + i], I.G32lo[go + i]);
            const int p1 = I.at_ptr[i + 1];
            for (int p = I.at_ptr[i]; p < p1; ++p) {
                const int4 a = ap[p];
                const float2 z = zin[a.x];
                ffc_mac(th, tl, __int_as_float(a.y), __int_as_float(a.z), z.x, z.y);
            }
            zout[i] = make_float2(th, tl);
        }
        __syncthreads();
    };
    {
        const float* sh = I.sig_ff + (size_t)(N - 1) * ns;
        const float* sl = sh + sx;
        const size_t go = (size_t)ldg * (c * nu + col);   // G_{N-1-c}
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            float th = 0.f, tl = 0.f;
            ffc_mac(th, tl, sh[i], sl[i], I.G32[go + i], I.G32lo[go + i]);
            z0[i] = make_float2(th, tl);
        }
        __syncthreads();
    }
    for (int d = N - 2 - c; d >= 0; --d) {
        step(z0, z1, d);
        float2* t = z0; z0 = z1; z1 = t;
    }
    const int nnzB = I.bc_ptr[nu];
    const float *bh = I.bc_ff, *bl = I.bc_ff + nnzB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c1 = c; c1 >= 0; --c1) {
        if (c1 < c) {
            step(z0, z1, -1);
            float2* t = z0; z0 = z1; z1 = t;
        }
        for (int a = warp; a < nu; a += nw) {
            float th = 0.f, tl = 0.f;
            for (int p = I.bc_ptr[a] + lane; p < I.bc_ptr[a + 1]; p += 32) {
                const float2 z = z0[I.bc_idx[p]];
                ffc_mac(th, tl, bh[p], bl[p], z.x, z.y);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, th, o), ol = __shfl_xor_sync(0xffffffffu, tl, o);
                const float s2 = th + oh;
                const float z = s2 - th;
                tl += ((th - (s2 - z)) + (oh - z)) + ol;
                th = s2;
            }
            if (lane == 0) {
                const int row = c1 * nu + a, cc = c * nu + col;
                double v = ((double)th + (double)tl) + I.H64[(size_t)row + (size_t)n * cc];
                if (row == cc) v = (v + I.sigu[row]) * (1.0 + shift);
                // within the diagonal block each pair is computed twice (by
                // the CTAs of both columns): the lower one is written to both
                if (c1 < c || row >= cc) I.M64[(size_t)row + (size_t)n * cc] = v;
                if (c1 < c || row > cc) I.M64[(size_t)cc + (size_t)n * row] = v;
            }
        }
    }
}

// Threads per chain CTA: the two z buffers take 16 ns bytes of shared memory,
// so a large ns leaves room for only one or two CTAs per SM; those get more
// threads (each thread owns fewer rows of z), so the SM keeps about 32 warps
// in flight to hide the latency of the sparse A' gathers and the FMA chains.
// The rows a thread owns change, not the arithmetic of any row: the result
// is the same bit for bit.
static int chain_threads(size_t smem) {
    const size_t per_sm = 227 * 1024;
    const size_t ctas = per_sm / (smem + 1024);
    return ctas >= 4 ? 256 : (ctas >= 2 ? 512 : 1024);
}

void launch_kkt_lyap_ff(const Inst* d_insts, int count, int max_ns, int max_nu, int max_N, int max_sx, int flags,
                        cudaStream_t st, double shift) {
    LQ_LAUNCH(lq_pdl(k_sig_split, dim3(per_instance_blocks(std::max(1, std::min(1024, (max_sx + 255) / 256)), count), count), 256, 0, st, d_insts, flags));
    const size_t smem = 2 * sizeof(float2) * (size_t)max_ns;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_ly_chain_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LQ_LAUNCH(lq_pdl(k_ly_chain_ff, dim3(max_N * max_nu, count), chain_threads(smem), smem, st, d_insts, flags, max_nu,
                                                                                           shift));
}

void launch_kkt_lyap(const Inst* d_insts, int count, int max_ns, int max_nu, int max_N, int flags,
                     cudaStream_t st, double shift) {
    const size_t smem = 2 * sizeof(double) * (size_t)max_ns;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_ly_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LQ_LAUNCH(lq_pdl(k_ly_chain, dim3(max_N * max_nu, count), chain_threads(smem), smem, st, d_insts, flags, max_nu,
                                                                                        shift));
}

// Multiply-add counts of the two ways to form Gamma' Sigma Gamma (the SYRK
// works on 64-wide tiles over the block triangle).
double kkt_cost_syrk(int ns, int nu, int N) {
    return (double)ns * nu * nu * N * (double)(N + 1) * (N + 2) / 6.0;
}

double kkt_cost_lyap(int ns, int nu, int N, long long nnzA, long long nnzB) {
    return (double)N * N * nu * (double)nnzA + 0.5 * N * (N + 1.0) * nu * (double)(ns + nnzB);
}

}  // namespace lqmpc
