// Iterative refinement of the mixed-precision KKT solve.
//
// M du = b is solved with the low-precision Cholesky factor; the residual
//     rho = b - (H du + Gamma'(Sigma_x (Gamma du)) + Sigma_u du)
// is evaluated matrix-free in FP64 (M itself is never formed in FP64), the
// correction solve uses the same factor, and the loop stops when
// ||rho||_inf <= refine_tol * ||b||_inf.  Every kernel is predicated on the
// instance flags, so a fixed launch sequence serves any number of steps.
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

__global__ void k_refine_begin(const Inst* __restrict__ insts) {
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    Scal* S = I.sc;
    if (S->done) return;
    double m = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) m = fmax(m, fabs(I.b[j]));
    m = block_reduce<1>(m, red);
    if (threadIdx.x == 0) {
        S->rnorm0 = m; S->rnorm = INFINITY; S->rnorm_prev = INFINITY;
        S->refine_ok = 0; S->refine_fail = 0; S->refine_cur = 0; S->stalled = 0;
    }
}

// rho_j = b_j - (H du)_j - mv_j - sigu_j du_j, mv = Gamma'(Sigma_x Gamma du).
// One warp per row; slot 6 partial = max |rho|.
__global__ void k_refine_resid(const Inst* __restrict__ insts, int du_role) {
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    const Scal* S = I.sc;
    if (S->done || S->refine_ok || S->refine_fail) return;
    const double* du = role_ptr(I, du_role);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double rmax = 0.0;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < I.n; j += gridDim.x * wpb) {
        const double* hc = I.H64 + (size_t)j * I.n;
        double acc = 0.0;
        for (int k = lane; k < I.n; k += 32) acc += hc[k] * du[k];
        acc = warp_sum(acc);
        if (lane == 0) {
            double r = I.b[j] - acc - I.mv[j] - I.sigu[j] * du[j];
            I.rho[j] = r;
            rmax = fmax(rmax, fabs(r));
        }
    }
    double v = block_reduce<1>(rmax, red);
    if (threadIdx.x == 0) I.part[6 * kMaxParts + blockIdx.x] = v;
}

__global__ void k_refine_check(const Inst* __restrict__ insts, int nb) {
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    Scal* S = I.sc;
    if (S->done || S->refine_ok || S->refine_fail) return;
    double m = 0.0;
    for (int p = threadIdx.x; p < nb; p += blockDim.x) m = fmax(m, I.part[6 * kMaxParts + p]);
    m = block_reduce<1>(m, red);
    if (threadIdx.x == 0) {
        S->rnorm = m;
        if (!(m == m)) { S->refine_fail = 1; return; }
        // converged: relative to ||b||, or small enough that the stationarity
        // residual it leaves behind is far below the stop tolerance
        const double floor_abs = 0.01 * S->tol * (1.0 + S->hnorm);
        if (m <= S->refine_tol * S->rnorm0 || m <= floor_abs || S->rnorm0 == 0.0) { S->refine_ok = 1; return; }
        if (m > 0.5 * S->rnorm_prev) S->stalled += 1;
        else S->stalled = 0;
        if (S->stalled >= 2) S->refine_fail = 1;
        S->rnorm_prev = m;
    }
}

__global__ void k_refine_update(const Inst* __restrict__ insts, int du_role, int last) {
    const Inst& I = insts[blockIdx.y];
    Scal* S = I.sc;
    if (S->done || S->refine_ok || S->refine_fail) return;
    double* du = role_ptr(I, du_role);
    if (!last)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < I.n; j += gridDim.x * blockDim.x)
            du[j] += I.dcorr[j];
    if (blockIdx.x == 0 && threadIdx.x == 0 && !last) {
        S->refine_cur += 1; S->refine_steps += 1; S->refine_iter += 1;
    }
}

// dst = src over the instance's SX (len_kind 0) or n (len_kind 1) entries.
__global__ void k_vec_copy(const Inst* __restrict__ insts, int src_role, int dst_role, int len_kind,
                           int force) {
    const Inst& I = insts[blockIdx.y];
    if (!force && I.sc->done) return;
    const double* s = role_ptr(I, src_role);
    double* d = role_ptr(I, dst_role);
    const int len = len_kind == 0 ? I.SX : I.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < len; k += gridDim.x * blockDim.x) d[k] = s[k];
}

static int nblk(int len, int th, int cap) {
    int b = (len + th - 1) / th;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

void launch_refine_begin(const Inst* d_insts, int count, int max_n, cudaStream_t st) {
    LQ_LAUNCH(k_refine_begin<<<dim3(1, count), 256, 0, st>>>(d_insts));
}

// one residual evaluation: rho = b - M du (needs tmpx = Gamma du and mv = Gamma'(Sigma tmpx))
void launch_refine_residual(const Inst* d_insts, int count, int max_n, cudaStream_t st) {
    int wpb = 8;
    int nb = nblk(max_n, wpb, kMaxParts);
    LQ_LAUNCH(k_refine_resid<<<dim3(nb, count), wpb * 32, 0, st>>>(d_insts, R_DU));
    LQ_LAUNCH(k_refine_check<<<dim3(1, count), 256, 0, st>>>(d_insts, nb));
}

void launch_refine_update(const Inst* d_insts, int count, int max_n, int last, cudaStream_t st) {
    LQ_LAUNCH(k_refine_update<<<dim3(nblk(max_n, 256, 1024), count), 256, 0, st>>>(d_insts, R_DU, last));
}

void launch_vec_copy(const Inst* d_insts, int count, int max_len, int src_role, int dst_role,
                     int len_kind, int force, cudaStream_t st) {
    LQ_LAUNCH(k_vec_copy<<<dim3(nblk(max_len, 256, 4096), count), 256, 0, st>>>(d_insts, src_role, dst_role,
                                                                                 len_kind, force));
}

}  // namespace lqmpc
