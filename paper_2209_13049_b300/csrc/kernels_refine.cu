// Accuracy recovery for the mixed-precision KKT solve: preconditioned
// conjugate gradients on M du = b (M symmetric positive definite, Eq. 7) with
// the low-precision Cholesky factor as preconditioner and every product with
// M evaluated matrix-free in FP64:
//     M p = H p + Gamma'(Sigma_x (Gamma p)) + Sigma_u p
// (M itself is never formed in FP64).  Started from x0 = Mlow^{-1} b, the
// first residual is that of plain iterative refinement; conjugate directions
// keep converging when the low-precision factor is too inaccurate for the
// stationary iteration to contract.  Gamma du is accumulated alongside
// (dxs += alpha Gamma p) so the step recovery needs no extra product.
//
// Stop: ||r||_inf <= refine_tol ||b||_inf, or <= 1e-4 res (1 + ||h||_inf) (the
// inexact-Newton forcing term, see pcg_test), or <= 0.01 tol (1 + ||h||_inf) (the
// stationarity residual left behind is then far below the stop test).
// Failure: a non-positive curvature p'Mp or a non-finite value.  Every kernel
// is predicated on the instance flags, so one launch sequence serves any
// number of steps and any batch.
#include "common.cuh"
#include "kernels.h"
#include "gamma_ff.cuh"

namespace lqmpc {

// `sel` is the launch predicate that picks the instances of this solve
// (pending, precision mask); refined or failed instances stop as well.
__device__ __forceinline__ bool pcg_skip(const Inst& I, int sel) {
    const Scal* S = I.sc;
    return skip_instance(I, sel) || S->refine_ok || S->refine_fail;
}

// Start: ||b||, flags cleared, step budget (BF16/TF32 factors get the low
// budget and FP32 factors the middle one: replacing such a factor by the next
// tier is cheaper than iterating with it).
__global__ void k_pcg_begin(const Inst* __restrict__ insts, int sel, int budget_hi, int budget_lo, int budget_mid) {
    pdl_wait();
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    Scal* S = I.sc;
    if (skip_instance(I, sel)) return;
    double m = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) m = fmax(m, fabs(I.b[j]));
    m = block_reduce<1>(m, red);
    if (threadIdx.x == 0) {
        S->rnorm0 = m; S->rnorm = INFINITY; S->rnorm_prev = INFINITY;
        S->refine_ok = 0; S->refine_fail = 0; S->refine_cur = 0; S->stalled = 0;
        S->refine_budget = (S->prec_cur == 1 || S->prec_cur == 2) ? budget_lo : (S->prec_cur == 3 ? budget_mid : budget_hi);
    }
}

// out_j = (H v)_j + mv_j + sigu_j v_j with mv = Gamma'(Sigma_x Gamma v); one
// warp per row.  mode 0 (initial residual): r = b - M du, partial max|r| in
// slot 6, and the last CTA runs the convergence test.  mode 1 (CG step):
// q = M p, partial p'q in slot 6, and the last CTA forms alpha.
__device__ void pcg_test(const Inst& I, double rn);
__device__ void pcg_alpha(const Inst& I, double pq);

__global__ void k_pcg_matvec(const Inst* __restrict__ insts, int mode, int sel) {
    pdl_wait();
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    if (pcg_skip(I, sel)) return;
    const double* v = mode == 0 ? I.du : I.pp;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    double acc_red = 0.0;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < I.n; j += gridDim.x * wpb) {
        const double* hc = I.H64 + (size_t)j * I.n;
        double acc = 0.0;
        for (int k = lane; k < I.n; k += 32) acc += hc[k] * v[k];
        acc = warp_sum(acc);
        if (lane == 0) {
            double mvj = acc + I.mv[j] + I.sigu[j] * v[j];
            if (mode == 0) {
                double r = I.b[j] - mvj;
                I.rho[j] = r;
                acc_red = fmax(acc_red, fabs(r));
            } else {
                I.qq[j] = mvj;
                acc_red += v[j] * mvj;
            }
        }
    }
    double t = mode == 0 ? block_reduce<1>(acc_red, red) : block_reduce<0>(acc_red, red);
    if (threadIdx.x == 0) I.part[6 * kMaxParts + blockIdx.x] = t;
    if (!last_arrival(I.sc)) return;
    double m = 0.0;
    for (int p = threadIdx.x; p < (int)gridDim.x; p += blockDim.x) {
        const double v = __ldcg(I.part + 6 * kMaxParts + p);
        m = mode == 0 ? fmax(m, v) : m + v;
    }
    m = mode == 0 ? block_reduce<1>(m, red) : block_reduce<0>(m, red);
    if (threadIdx.x == 0) {
        if (mode == 0) pcg_test(I, m);
        else pcg_alpha(I, m);
    }
}

// k_pcg_matvec with mv_j gathered from the float-float Gamma' partials (no
// separate sum launch).  Eight warps per CTA, WPR warps per row: the group's
// threads split the row of H (its loads in flight at once: four per thread)
// and its warps split the Gamma' partials, and the warps' sums meet in shared
// memory.  A single instance takes a whole CTA per row (WPR = 8: a row costs
// about one round trip to L2); a batch, whose instances get few CTAs each,
// one warp per row (WPR = 1: eight rows per CTA in flight).  In the
// conjugate-gradient steps the last CTA's tail also leaves nothing else to
// do: alpha is formed there as in k_pcg_matvec.
constexpr int kMvThreads = 256, kMvH = 4;
template <int WPR>
__global__ void __launch_bounds__(kMvThreads) k_pcg_matvec_ff(const Inst* __restrict__ insts, int mode, int sel,
                                                              int splits) {
    pdl_wait();
    constexpr int kW = kMvThreads / 32, RPC = kW / WPR, GT = 32 * WPR;
    __shared__ float2 wsum[kW];
    __shared__ double gred[RPC];
    __shared__ double fin[1];
    const Inst& I = insts[blockIdx.y];
    if (pcg_skip(I, sel)) return;
    const double* v = mode == 0 ? I.du : I.pp;
    const int n = I.n, N = I.N, nu = I.nu, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = warp / WPR, wg = warp % WPR, tg = wg * 32 + lane;   // row group, warp and thread in it
    const size_t stride = (size_t)N * n;          // one split's partials
    double acc_red = 0.0;                          // the group leader's
    for (int j0 = blockIdx.x * RPC; j0 < n; j0 += gridDim.x * RPC) {   // uniform trip count in the CTA
        const int j = j0 + grp;
        double s = 0.0;               // this lane's share of H row j . v (FP64)
        float gh = 0.f, gl = 0.f;     // and of the Gamma' partials (float-float)
        if (j < n) {
            const double* hc = I.H64 + (size_t)j * n;
            double hv[kMvH], vv[kMvH];
#pragma unroll
            for (int u = 0; u < kMvH; ++u) {
                const int k = tg + GT * u;
                hv[u] = k < n ? hc[k] : 0.0;
                vv[u] = k < n ? v[k] : 0.0;
            }
            // Gamma' partials of output j (see gamma_tmv_ff_gather)
            const int t = j / nu, c = j % nu, nd = N - t;
            const float2* base = ff_parts(I) + ((size_t)t * nu + c) * N;
            constexpr int QS = kFfMaxSplits / WPR;
            float2 g[2 * QS];
#pragma unroll
            for (int q = 0; q < QS; ++q) {
                const int sp = wg + WPR * q;
                const float2* src = base + (size_t)sp * stride;
                g[2 * q] = (sp < splits && lane < nd) ? src[lane] : make_float2(0.f, 0.f);
                g[2 * q + 1] = (sp < splits && lane + 32 < nd) ? src[lane + 32] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kMvH; ++u) s = fma(hv[u], vv[u], s);
            for (int k = tg + GT * kMvH; k < n; k += GT) s = fma(hc[k], v[k], s);
#pragma unroll
            for (int q = 0; q < 2 * QS; ++q) ff_acc(gh, gl, g[q].x, g[q].y);
            for (int sp = wg; sp < splits; sp += WPR)
                for (int d = lane + 64; d < nd; d += 32) {
                    const float2 p = base[(size_t)sp * stride + d];
                    ff_acc(gh, gl, p.x, p.y);
                }
        }
        // the lane's H v share joins the float-float sum, and the lanes' and
        // warps' sums meet on the FP32 pipe (FP64 adds issue at two lanes per
        // clock per SM); one conversion back to FP64 per row
        {
            float h, l;
            split_ff(s, h, l);
            ff_acc(gh, gl, h, l);
        }
        warp_sum_ff(gh, gl);
        if (WPR > 1) {
            if (lane == 0) wsum[warp] = make_float2(gh, gl);
            __syncthreads();
            if (tg == 0) {
                float mh = 0.f, ml = 0.f;
#pragma unroll
                for (int w = 0; w < WPR; ++w) ff_acc(mh, ml, wsum[grp * WPR + w].x, wsum[grp * WPR + w].y);
                gh = mh;
                gl = ml;
            }
            __syncthreads();
        }
        s = (double)gh + (double)gl;
        if (tg == 0 && j < n) {
            const double mj = s + I.sigu[j] * v[j];
            if (mode == 0) {
                const double r = I.b[j] - mj;
                I.rho[j] = r;
                acc_red = max_nonneg(acc_red, fabs(r));
            } else {
                I.qq[j] = mj;
                acc_red += v[j] * mj;
            }
        }
    }
    // The CTA's partial: only the row groups' leaders hold values (one per
    // group), so they meet in shared memory and thread 0 combines them in
    // group order -- no block-wide FP64 shuffle tree.
    if (tg == 0) gred[grp] = acc_red;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = gred[0];
        for (int q = 1; q < RPC; ++q) t = mode == 0 ? max_nonneg(t, gred[q]) : t + gred[q];
        I.part[6 * kMaxParts + blockIdx.x] = t;
    }
    if (!last_arrival(I.sc)) return;
    {
        constexpr int slot[1] = {6};
        const int kind[1] = {mode == 0 ? (int)kMaxNonneg : (int)kSum};
        const int cnt[1] = {(int)gridDim.x};
        reduce_parts<1>(I, slot, kind, cnt, fin);
    }
    if (threadIdx.x == 0) {
        if (mode == 0) pcg_test(I, fin[0]);
        else pcg_alpha(I, fin[0]);
    }
}

// Convergence test on the residual norm.  Besides the relative and absolute
// tolerances, an inexact-Newton forcing term: the residual of the Newton
// system need only be small next to the interior-point residual it is to
// reduce, ||r|| <= 1e-4 res (1 + ||h||) with res = max(res_d, res_p, mu) of
// the current iterate (zero outside an interior-point solve).  Early
// iterations then stop at the preconditioner's own solution; as res falls
// to the stop tolerance this meets the absolute floor.
constexpr double kForcing = 1e-4;
constexpr int kProjectAfter = 8;   // steps before the contraction rate is trusted
__device__ void pcg_test(const Inst& I, double rn) {
    Scal* S = I.sc;
    S->rnorm = rn;
    if (!(rn == rn)) { S->refine_fail = 1; return; }
    const double scale = 1.0 + S->hnorm;
    const double floor_abs = 0.01 * S->tol * scale;
    const double forcing = kForcing * S->res * scale;
    const double target = fmax(S->refine_tol * S->rnorm0, fmax(floor_abs, forcing));
    if (rn <= target || S->rnorm0 == 0.0) {
        S->refine_ok = 1;
    } else if (S->refine_cur >= S->refine_budget) {
        S->refine_fail = 1;
    } else if (S->refine_cur >= kProjectAfter) {
        // Hopeless runs stop early: at the mean contraction so far the
        // target would take more than the step budget.
        const double k = S->refine_cur, got = log(rn / S->rnorm0);
        const double need = got < 0.0 ? k * log(target / rn) / got : INFINITY;
        if (k + need > S->refine_budget) S->refine_fail = 1;
    }
}

// Control of the device-side conjugate-gradient loop (the while node of a
// captured graph): go on while some selected instance's refinement is
// neither converged nor failed (nor its factor failed), for at most `cap`
// passes.  reset: the pass count restarts (the launch after the initial
// residual).  The pass count is left in instance 0's Scal for the host.
__global__ void k_pcg_more(const Inst* __restrict__ insts, int count, int selr, cudaGraphConditionalHandle h,
                           int cap, int reset, int slot) {
    pdl_wait();
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < count; q += blockDim.x) {
        const Inst& I = insts[q];
        if (!skip_instance(I, selr) && !I.sc->info) atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* loops = insts[0].bar + 4;
        const unsigned k = reset ? 0u : *loops + 1u;
        *loops = k;
        insts[0].sc->pcg_loops = (int)k;
        if (!reset) insts[0].sc->pcg_pass_total[slot] += 1;
        cudaGraphSetConditional(h, (any && k < (unsigned)cap) ? 1u : 0u);
    }
}

void launch_pcg_more(const Inst* d_insts, int count, int selr, cudaGraphConditionalHandle h, int cap, int reset,
                     int slot, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_pcg_more, 1, 256, 0, st, d_insts, count, selr, h, cap, reset, slot));
}

// p = z, rz = r'z (one block per instance).
__global__ void k_pcg_pinit(const Inst* __restrict__ insts, int sel) {
    pdl_wait();
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    if (pcg_skip(I, sel)) return;
    double s = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        I.pp[j] = I.dcorr[j];
        s += I.rho[j] * I.dcorr[j];
    }
    s = block_reduce<0>(s, red);
    if (threadIdx.x == 0) I.sc->pcg_rz = s;
}

// alpha = r'z / p'Mp; a non-positive curvature marks failure.
__device__ void pcg_alpha(const Inst& I, double pq) {
    Scal* S = I.sc;
    if (!(pq > 0.0) || !(S->pcg_rz == S->pcg_rz)) { S->refine_fail = 1; return; }
    S->pcg_alpha = S->pcg_rz / pq;
    S->refine_cur += 1; S->refine_steps += 1; S->refine_iter += 1;
}

// du += alpha p, r -= alpha q (input rows), dxs += alpha (Gamma p) (state
// rows).  Partial max|r| in slot 7; the last CTA runs the convergence test.
__global__ void k_pcg_axpy(const Inst* __restrict__ insts, int sel) {
    pdl_wait();
    __shared__ long long ext[32];
    __shared__ double fin[1];
    const Inst& I = insts[blockIdx.y];
    if (pcg_skip(I, sel)) return;
    const double al = I.sc->pcg_alpha;
    const int total = I.SX + I.n;
    long long rmax = 0;   // bits of max |r| (integer order, no FP64 max)
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        if (k < I.n) {
            I.du[k] += al * I.pp[k];
            double r = I.rho[k] - al * I.qq[k];
            I.rho[k] = r;
            const long long a = abs_bits(r);
            rmax = a > rmax ? a : rmax;
        } else {
            const int q = k - I.n;
            I.dxs[q] += al * I.tmpx[q];
        }
    }
    double v = block_ext<true>(rmax, ext);
    if (threadIdx.x == 0) I.part[7 * kMaxParts + blockIdx.x] = v;
    if (!last_arrival(I.sc)) return;
    {
        constexpr int slot[1] = {7}, kind[1] = {kMaxNonneg};
        const int cnt[1] = {(int)gridDim.x};
        reduce_parts<1>(I, slot, kind, cnt, fin);
    }
    if (threadIdx.x == 0) pcg_test(I, fin[0]);
}

// beta = r'z_new / r'z_old; p = z + beta p (one block per instance).
__global__ void k_pcg_beta(const Inst* __restrict__ insts, int sel) {
    pdl_wait();
    __shared__ double red[32];
    __shared__ double beta_sh;
    const Inst& I = insts[blockIdx.y];
    Scal* S = I.sc;
    if (pcg_skip(I, sel)) return;
    double s = 0.0;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) s += I.rho[j] * I.dcorr[j];
    s = block_reduce<0>(s, red);
    if (threadIdx.x == 0) {
        beta_sh = S->pcg_rz != 0.0 ? s / S->pcg_rz : 0.0;
        S->pcg_rz = s;
    }
    __syncthreads();
    const double be = beta_sh;
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) I.pp[j] = I.dcorr[j] + be * I.pp[j];
}

// dst = src over the instance's SX (len_kind 0) or n (len_kind 1) entries.
__global__ void k_vec_copy(const Inst* __restrict__ insts, int src_role, int dst_role, int len_kind,
                           int flags) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags)) return;
    const double* s = role_ptr(I, src_role);
    double* d = role_ptr(I, dst_role);
    const int len = len_kind == 0 ? I.SX : I.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < len; k += gridDim.x * blockDim.x) d[k] = s[k];
}

// dst += src over the instance's n entries (instances not done).
// Every unfinished instance needs a KKT solve.
__global__ void k_kkt_begin(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.x];
    // an instance whose predictor failed unseen (spec_fail) skips the corrector
    if (threadIdx.x == 0) I.sc->kkt_pending = (I.sc->done || I.sc->spec_fail) ? 0 : 1;
}

// Settle the pending KKT solves: an FP64 solve that met no failing pivot (a
// refinement of it that did not converge keeps its best iterate), or a
// low-precision one whose refinement converged.  The rest stay pending for
// the host: escalation to a more accurate factor, or a final status.  With
// `mark` (the host reads the outcome only at the end of the iteration) a
// solve left pending also sets spec_fail, so that the iteration's step and
// update are skipped.
__global__ void k_kkt_settle(const Inst* __restrict__ insts, int mark) {
    pdl_wait();
    const Inst& I = insts[blockIdx.x];
    Scal* S = I.sc;
    if (threadIdx.x != 0 || S->done || !S->kkt_pending) return;
    if (!S->info && (S->prec_cur == 0 || S->refine_ok)) S->kkt_pending = 0;
    else if (mark) S->spec_fail = 1;
}

__global__ void k_vec_add(const Inst* __restrict__ insts, int src_role, int dst_role) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done) return;
    const double* s = role_ptr(I, src_role);
    double* d = role_ptr(I, dst_role);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < I.n; k += gridDim.x * blockDim.x) d[k] += s[k];
}

static int nblk(int len, int th, int cap) {
    int b = (len + th - 1) / th;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

void launch_pcg_begin(const Inst* d_insts, int count, int sel, int budget_hi, int budget_lo, int budget_mid,
                      cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_pcg_begin, dim3(1, count), 256, 0, st, d_insts, sel, budget_hi, budget_lo, budget_mid));
}

// mode 0: r = b - M du and its convergence test; mode 1: q = M p and alpha.
void launch_pcg_matvec(const Inst* d_insts, int count, int max_n, int mode, int sel, cudaStream_t st) {
    int wpb = 8;
    int nb = nblk(max_n, wpb, kMaxParts);
    LQ_LAUNCH(lq_pdl(k_pcg_matvec, dim3(nb, count), wpb * 32, 0, st, d_insts, mode, sel));
}

void launch_pcg_matvec_ff(const Inst* d_insts, int count, int max_n, int splits, int mode, int sel,
                          cudaStream_t st) {
    if (count == 1) {   // a CTA per row
        const int nb = nblk(max_n, 1, kMaxParts);
        LQ_LAUNCH(lq_pdl(k_pcg_matvec_ff<8>, dim3(nb, count), kMvThreads, 0, st, d_insts, mode, sel, splits));
    } else {            // a warp per row
        const int nb = per_instance_blocks(nblk(max_n, kMvThreads / 32, kMaxParts), count);
        LQ_LAUNCH(lq_pdl(k_pcg_matvec_ff<1>, dim3(nb, count), kMvThreads, 0, st, d_insts, mode, sel, splits));
    }
}

void launch_pcg_pinit(const Inst* d_insts, int count, int sel, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_pcg_pinit, dim3(1, count), 256, 0, st, d_insts, sel));
}

void launch_pcg_step_update(const Inst* d_insts, int count, int max_total, int sel, cudaStream_t st) {
    int nb = per_instance_blocks(nblk(max_total, 256, kMaxParts), count);
    LQ_LAUNCH(lq_pdl(k_pcg_axpy, dim3(nb, count), 256, 0, st, d_insts, sel));
}

void launch_pcg_beta(const Inst* d_insts, int count, int sel, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_pcg_beta, dim3(1, count), 256, 0, st, d_insts, sel));
}

void launch_vec_copy(const Inst* d_insts, int count, int max_len, int src_role, int dst_role,
                     int len_kind, int force, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_vec_copy, dim3(nblk(max_len, 256, 4096), count), 256, 0, st, d_insts, src_role, dst_role,
                                                                                 len_kind, force));
}

void launch_vec_add(const Inst* d_insts, int count, int max_n, int src_role, int dst_role, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_vec_add, dim3(nblk(max_n, 256, 1024), count), 256, 0, st, d_insts, src_role, dst_role));
}

void launch_kkt_begin(const Inst* d_insts, int count, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_kkt_begin, count, 32, 0, st, d_insts));
}

void launch_kkt_settle(const Inst* d_insts, int count, cudaStream_t st, int mark) {
    LQ_LAUNCH(lq_pdl(k_kkt_settle, count, 32, 0, st, d_insts, mark));
}

}  // namespace lqmpc
