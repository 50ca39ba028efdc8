// FP64 condensed KKT matrix (Eq. 7) by a backward recursion over the
// horizon instead of the SYRK, for plants whose A is sparse.
//
// With Gamma's blocks A^k B (Section II), block (c1, c) of Gamma' Sigma_x
// Gamma for c1 <= c is
//     sum_{r >= c} (A^{r-c1} B)' Sigma_r A^{r-c} B = (A^{c-c1} B)' P_c B,
//     P_c = sum_{r >= c} (A^{r-c})' Sigma_r A^{r-c},
// and P satisfies P_{N-1} = Sigma_{N-1}, P_c = Sigma_c + A' P_{c+1} A.  So the
// matrix costs N products A' P A with a sparse A (2 nnz(A) ns multiply-adds
// each) plus the blocks G_d' W_c with W_c = P_c B, instead of the SYRK's
// ns nu^2 N^3 / 6: about 3x fewer FP64 operations for the 2-D heat plants
// (FP64 runs at 1/64 of the FP32 rate on this part).  The same matrix up to
// rounding order.
//
// Layout: P and T are ns x ns column-major FP64; W holds W_c for every stage
// (N x ns x nu).  A' is available as CSR (the columns of A); B's nonzeros as
// per-column lists.  For batches the stage loop runs over the largest horizon
// and instance q uses its own stage c = N_q - 1 - g.
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

// g = 0: P = diag(Sigma_{N-1}).
__global__ void k_ly_init(const Inst* __restrict__ insts, int flags) {
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || !I.lyP) return;
    const int ns = I.ns;
    const double* sg = I.sigx + (size_t)(I.N - 1) * ns;
    const size_t total = (size_t)ns * ns;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % ns), j = (int)(q / ns);
        I.lyP[q] = i == j ? sg[i] : 0.0;
    }
}

// T = P A: T[:, j] = sum over the nonzeros A[k, j] of P[:, k] A[k, j].
__global__ void k_ly_pa(const Inst* __restrict__ insts, int flags, int g) {
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || !I.lyP || I.N - 1 - g < 0) return;
    const int ns = I.ns;
    const size_t total = (size_t)ns * ns;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % ns), j = (int)(q / ns);
        double acc = 0.0;
        for (int p = I.at_ptr[j]; p < I.at_ptr[j + 1]; ++p) acc += I.lyP[i + (size_t)ns * I.at_idx[p]] * I.at_val[p];
        I.lyT[q] = acc;
    }
}

// P = A' T + diag(Sigma_c): P[i, j] = sum over the nonzeros A[k, i] of A[k, i] T[k, j].
__global__ void k_ly_atp(const Inst* __restrict__ insts, int flags, int g) {
    const Inst& I = insts[blockIdx.y];
    const int c = I.N - 1 - g;
    if (skip_instance(I, flags) || !I.lyP || c < 0) return;
    const int ns = I.ns;
    const double* sg = I.sigx + (size_t)c * ns;
    const size_t total = (size_t)ns * ns;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % ns), j = (int)(q / ns);
        double acc = i == j ? sg[i] : 0.0;
        for (int p = I.at_ptr[i]; p < I.at_ptr[i + 1]; ++p) acc += I.at_val[p] * I.lyT[I.at_idx[p] + (size_t)ns * j];
        I.lyP[q] = acc;
    }
}

// W_c = P_c B from B's per-column nonzero lists.
__global__ void k_ly_w(const Inst* __restrict__ insts, int flags, int g) {
    const Inst& I = insts[blockIdx.y];
    const int c = I.N - 1 - g;
    if (skip_instance(I, flags) || !I.lyP || c < 0) return;
    const int ns = I.ns, nu = I.nu;
    double* W = I.lyW + (size_t)c * ns * nu;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ns * nu; q += gridDim.x * blockDim.x) {
        const int i = q % ns, b = q / ns;
        double acc = 0.0;
        for (int p = I.bc_ptr[b]; p < I.bc_ptr[b + 1]; ++p) acc += I.lyP[i + (size_t)ns * I.bc_idx[p]] * I.bc_val[p];
        W[q] = acc;
    }
}

// M = H + [G_{c-c1}' W_c] + diag(Sigma_u): one block (c1 <= c) per CTA,
// nu x nu outputs over the threads, states strided; both triangles written.
__global__ void k_ly_assemble(const Inst* __restrict__ insts, int flags, double shift) {
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || !I.lyP) return;
    const int ns = I.ns, nu = I.nu, N = I.N, n = I.n;
    const int npairs = N * (N + 1) / 2;
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        int c = 0;
        while ((c + 1) * (c + 2) / 2 <= pr) ++c;
        const int c1 = pr - c * (c + 1) / 2;    // c1 <= c
        const int d = c - c1;
        const double* W = I.lyW + (size_t)c * ns * nu;
        for (int o = threadIdx.x; o < nu * nu; o += blockDim.x) {
            const int a = o % nu, b = o / nu;
            const double* Ga = I.G64 + (size_t)I.ldg * ((N - 1 - d) * nu + a);
            const double* Wb = W + (size_t)b * ns;
            double acc = 0.0;
            for (int i = 0; i < ns; ++i) acc += Ga[i] * Wb[i];
            const int row = c1 * nu + a, col = c * nu + b;
            double v = acc + I.H64[(size_t)row + (size_t)n * col];
            if (row == col) v = (v + I.sigu[row]) * (1.0 + shift);   // shift: a retried factor
            I.M64[(size_t)row + (size_t)n * col] = v;
            if (row != col) I.M64[(size_t)col + (size_t)n * row] = v;
        }
    }
}

static int ly_blocks(size_t work) {
    size_t b = (work + 255) / 256;
    return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

void launch_kkt_lyap(const Inst* d_insts, int count, int max_ns, int max_nu, int max_N, int flags,
                     cudaStream_t st, double shift) {
    const size_t sq = (size_t)max_ns * max_ns;
    LQ_LAUNCH(k_ly_init<<<dim3(ly_blocks(sq), count), 256, 0, st>>>(d_insts, flags));
    LQ_LAUNCH(k_ly_w<<<dim3(ly_blocks((size_t)max_ns * max_nu), count), 256, 0, st>>>(d_insts, flags, 0));
    for (int g = 1; g < max_N; ++g) {
        LQ_LAUNCH(k_ly_pa<<<dim3(ly_blocks(sq), count), 256, 0, st>>>(d_insts, flags, g));
        LQ_LAUNCH(k_ly_atp<<<dim3(ly_blocks(sq), count), 256, 0, st>>>(d_insts, flags, g));
        LQ_LAUNCH(k_ly_w<<<dim3(ly_blocks((size_t)max_ns * max_nu), count), 256, 0, st>>>(d_insts, flags, g));
    }
    const int npairs = max_N * (max_N + 1) / 2;
    LQ_LAUNCH(k_ly_assemble<<<dim3(npairs < 4096 ? npairs : 4096, count), 128, 0, st>>>(d_insts, flags, shift));
}

// Multiply-add counts of the two ways to form Gamma' Sigma Gamma (the SYRK
// works on 64-wide tiles over the block triangle).
double kkt_cost_syrk(int ns, int nu, int N) {
    return (double)ns * nu * nu * N * (double)(N + 1) * (N + 2) / 6.0;
}

double kkt_cost_lyap(int ns, int nu, int N, long long nnzA, long long nnzB) {
    return (double)N * (2.0 * (double)nnzA * ns + (double)nnzB * ns) + 0.5 * N * (N + 1.0) * nu * nu * ns;
}

}  // namespace lqmpc
