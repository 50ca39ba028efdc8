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
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

__global__ void k_ly_chain(const Inst* __restrict__ insts, int flags, int max_nu, double shift) {
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
                I.M64[(size_t)row + (size_t)n * cc] = v;
                if (c1 < c) I.M64[(size_t)cc + (size_t)n * row] = v;
            }
        }
        // the next step overwrites the other buffer only; the dots above read
        // z0, which the step after it overwrites behind a barrier
    }
}

void launch_kkt_lyap(const Inst* d_insts, int count, int max_ns, int max_nu, int max_N, int flags,
                     cudaStream_t st, double shift) {
    const size_t smem = 2 * sizeof(double) * (size_t)max_ns;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_ly_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    LQ_LAUNCH(k_ly_chain<<<dim3(max_N * max_nu, count), 256, smem, st>>>(d_insts, flags, max_nu, shift));
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
