// Interior-point vector kernels: initial point, residuals and Sigma, Mehrotra
// predictor/corrector right-hand sides, fraction-to-boundary step lengths and
// the iterate update (Section III, Eqs. 5-7 and Algorithm 1).
//
// Notation.  The dense QP (Eq. 3) has variables u (n = nu*N) and the
// constraint J u <= d with J = [Gamma; -Gamma; I; -I]: four families of
// one-sided rows, each with a slack s and a dual z:
//   family 1 (state upper):  x + s1 = xu     family 2 (state lower): -x + s2 = -xl
//   family 3 (input upper):  u + s3 = uu     family 4 (input lower): -u + s4 = -ul
// where x = Phi xbar + Gamma u is kept as an iterate.  A two-sided row is one
// row of Gamma with two slacks.  Rows whose bound is infinite are absent:
// their s = 1, z = 0 never change and they are left out of every sum.
//
// Reductions are deterministic: every block writes one partial per slot, and
// the finish combines them in a fixed order.
//
// The per-row arithmetic is FP64, and the FP64 pipe of this part is narrow
// (two lanes per clock per SM): these kernels are bound by the FP64
// instructions of their most loaded SM.  Hence an equal share of rows per SM
// (ew_grid), the primal residual, the reciprocal slacks and the corrector's
// r_c formed once per iteration and loaded by the later kernels (a division
// is some ten FP64 instructions), and reductions that leave the FP64 pipe
// alone where they can (put_parts, reduce_parts: one warp per quantity, so
// the finish in the instance's last CTA, while the other SMs wait, is one
// round of loads and one barrier).
#include "common.cuh"
#include "gamma_ff.cuh"
#include "kernels.h"

namespace lqmpc {

// ---------------------------------------------------------------------------
// Per-row helpers
// ---------------------------------------------------------------------------

struct RowView {
    double* s_u; double* z_u; double* s_l; double* z_l;   // upper / lower slack, dual
    double* ds_u; double* dz_u; double* ds_l; double* dz_l;
    double lo, hi;        // bounds of this row
    double v;             // current value (x_k or u_j)
    bool fu, fl;          // bounds finite
};

// isfinite on the bit pattern (integer pipe)
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double_as_longlong(x) & 0x7FF0000000000000LL) != 0x7FF0000000000000LL;
}

__device__ __forceinline__ RowView row_view(const Inst& I, int k) {
    RowView r;
    if (k < I.SX) {
        int i = k % I.ns;
        r.s_u = I.s1 + k; r.z_u = I.z1 + k; r.s_l = I.s2 + k; r.z_l = I.z2 + k;
        r.ds_u = I.ds1 + k; r.dz_u = I.dz1 + k; r.ds_l = I.ds2 + k; r.dz_l = I.dz2 + k;
        r.lo = I.xl[i]; r.hi = I.xu[i]; r.v = I.x[k];
    } else {
        int j = k - I.SX, c = j % I.nu;
        r.s_u = I.s3 + j; r.z_u = I.z3 + j; r.s_l = I.s4 + j; r.z_l = I.z4 + j;
        r.ds_u = I.ds3 + j; r.dz_u = I.dz3 + j; r.ds_l = I.ds4 + j; r.dz_l = I.dz4 + j;
        r.lo = I.ul[c]; r.hi = I.uu[c]; r.v = I.u[j];
    }
    r.fu = finite_bits(r.hi); r.fl = finite_bits(r.lo);
    return r;
}

constexpr int kEwMaxThreads = 1024;   // largest CTA of the per-row kernels

// Write one partial per slot for this block.
__device__ __forceinline__ void put_part(const Inst& I, int slot, double v) {
    if (threadIdx.x == 0) I.part[slot * kMaxParts + blockIdx.x] = v;
}

// ---------------------------------------------------------------------------
// Initial point.  u0 = box midpoint (lo+1 / hi-1 for one-sided boxes, 0 for
// none); x0 = y + Gamma u0 (Gamma u0 precomputed into tmpx); s0 = max(slack, 1)
// and z0 = 1 for present rows.  The warm start replaces u0 by a clipped guess
// and z0 by mu0 / s0.  Also the norms ||d|| and ||h|| of the stop
// test and the row count m.
// ---------------------------------------------------------------------------

__global__ void k_set_u0(const Inst* __restrict__ insts, int warm) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < I.n; j += gridDim.x * blockDim.x) {
        int c = j % I.nu;
        double lo = I.ul[c], hi = I.uu[c];
        bool fl = isfinite(lo), fh = isfinite(hi);
        if (!warm) {
            I.u[j] = (fl && fh) ? 0.5 * (lo + hi) : fl ? lo + 1.0 : fh ? hi - 1.0 : 0.0;
        } else {
            // warm start: the guess (staged in du_aff) clipped into the box with
            // a margin of 1% of a two-sided range, 1e-2 for a one-sided bound
            const double g = I.du_aff[j];
            const double mg = (fl && fh) ? 0.01 * (hi - lo) : 0.01;
            double v = g;
            if (fl) v = fmax(v, lo + mg);
            if (fh) v = fmin(v, hi - mg);
            if (fl && fh && hi - lo <= 2.0 * mg) v = 0.5 * (lo + hi);
            I.u[j] = v;
        }
    }
}

// Cold start: s = max(slack, 1), z = 1.  Warm start (mu0 > 0): s =
// max(slack, smin), z = mu0 / s, a start centred at complementarity mu0.
__global__ void k_init_slacks(const Inst* __restrict__ insts, double mu0, double smin) {
    pdl_wait();
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    const bool warm = mu0 > 0.0;
    const double sfloor = warm ? smin : 1.0;
    auto zof = [&](double sv) { return warm ? mu0 / sv : 1.0; };
    const int total = I.SX + I.n;
    double cnt = 0.0, dmax = 0.0, hmax = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        if (k < I.SX) {
            int i = k % I.ns;
            double xk = I.y[k] + I.tmpx[k];
            I.x[k] = xk;
            double hi = I.xu[i], lo = I.xl[i];
            bool fu = isfinite(hi), fl = isfinite(lo);
            I.s1[k] = fu ? fmax(hi - xk, sfloor) : 1.0; I.z1[k] = fu ? zof(I.s1[k]) : 0.0;
            I.s2[k] = fl ? fmax(xk - lo, sfloor) : 1.0; I.z2[k] = fl ? zof(I.s2[k]) : 0.0;
            cnt += (double)fu + (double)fl;
            double yk = I.y[k];
            if (fu) dmax = fmax(dmax, fabs(hi - yk));
            if (fl) dmax = fmax(dmax, fabs(yk - lo));
        } else {
            int j = k - I.SX, c = j % I.nu;
            double uj = I.u[j], hi = I.uu[c], lo = I.ul[c];
            bool fu = isfinite(hi), fl = isfinite(lo);
            I.s3[j] = fu ? fmax(hi - uj, sfloor) : 1.0; I.z3[j] = fu ? zof(I.s3[j]) : 0.0;
            I.s4[j] = fl ? fmax(uj - lo, sfloor) : 1.0; I.z4[j] = fl ? zof(I.s4[j]) : 0.0;
            cnt += (double)fu + (double)fl;
            if (fu) dmax = fmax(dmax, fabs(hi));
            if (fl) dmax = fmax(dmax, fabs(lo));
            hmax = fmax(hmax, fabs(I.h[j]));
        }
    }
    double v = block_reduce<0>(cnt, red); put_part(I, 0, v);
    v = block_reduce<1>(dmax, red); put_part(I, 1, v);
    v = block_reduce<1>(hmax, red); put_part(I, 2, v);
}

__global__ void k_init_fin(const Inst* __restrict__ insts, int nparts, double tol, double tau,
                           int max_iter, double refine_tol, int prec) {
    pdl_wait();
    __shared__ double red[32];
    const Inst& I = insts[blockIdx.y];
    double c = 0, d = 0, h = 0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
        c += I.part[0 * kMaxParts + p];
        d = fmax(d, I.part[1 * kMaxParts + p]);
        h = fmax(h, I.part[2 * kMaxParts + p]);
    }
    c = block_reduce<0>(c, red);
    d = block_reduce<1>(d, red);
    h = block_reduce<1>(h, red);
    if (threadIdx.x == 0) {
        Scal* S = I.sc;
        S->m = (int)(c + 0.5);
        S->dnorm = d; S->hnorm = h;
        S->tol = tol; S->tau = tau; S->max_iter = max_iter; S->refine_tol = refine_tol;
        S->done = 0; S->status = 0; S->iter = 0; S->info = 0;
        S->refine_steps = 0; S->fallbacks = 0; S->use_fp64 = 0; S->err = 0;
        S->mu = S->sigma = S->alpha = S->alpha_aff = 0.0;
        S->prec_cur = prec; S->kkt_pending = 0; S->refine_budget = 0;
    }
}

// ---------------------------------------------------------------------------
// Residuals (Eq. 5), Sigma = S^{-1} Z (Eq. 6) and the predictor vectors.
//   r_p per family (kept in rpu / rpl for the step kernels of the iteration),
//   1/s per family (rsu / rsl), Sigma_x = z1/s1 + z2/s2 per state row,
//   Sigma_u likewise (z/s of each family in sgu / sgl); wz = z1 - z2 (for
//   the Gamma' z term of r_d);
//   predictor w_i = z_i - Sigma_i r_p,i, combined wx = w1 - w2 (for Gamma').
// Partials: slot 0 max|r_p|, slot 1 sum s.z.  With split, also the
// float-float split of wz and wx for the float-float Gamma' product of both
// (hi0, lo0, hi1, lo1 in ffw: no split launch).
// ---------------------------------------------------------------------------

__global__ void k_resid(const Inst* __restrict__ insts, int split) {
    pdl_wait();
    __shared__ double stage[2 * kEwMaxThreads];
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done) return;
    // An iteration starts with no failed solve and no failed pivot (a repeat
    // of an iteration whose solve failed unseen starts afresh); the first
    // kernel of the iteration on the main stream, before any KKT launch.
    if (blockIdx.x == 0 && threadIdx.x == 0) { I.sc->spec_fail = 0; I.sc->info = 0; }
    const int total = I.SX + I.n;
    long long rpmax = 0;   // bits of max |r_p|
    double sz = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        RowView r = row_view(I, k);
        double su = *r.s_u, zu = *r.z_u, sl = *r.s_l, zl = *r.z_l;
        double rpu = r.fu ? r.v + su - r.hi : 0.0;
        double rpl = r.fl ? -r.v + sl + r.lo : 0.0;
        // 1/s once per iteration: Sigma here, the corrector and the step
        // multiply by it (an absent row has s = 1, z = 0)
        const double rsu = 1.0 / su, rsl = 1.0 / sl;
        const double sgu = zu * rsu, sgl = zl * rsl;
        I.sgu[k] = sgu; I.sgl[k] = sgl;
        I.rsu[k] = rsu; I.rsl[k] = rsl;
        I.rpu[k] = rpu; I.rpl[k] = rpl;
        const long long a = abs_bits(rpu), b = abs_bits(rpl);
        rpmax = a > rpmax ? a : rpmax;
        rpmax = b > rpmax ? b : rpmax;
        if (r.fu) sz += su * zu;
        if (r.fl) sz += sl * zl;
        double wz = zu - zl;
        double wx = (zu - sgu * rpu) - (zl - sgl * rpl);
        if (k < I.SX) {
            I.sigx[k] = sgu + sgl; I.sigx32[(size_t)(k / I.ns) * I.ldg + k % I.ns] = (float)(sgu + sgl);
            I.wz[k] = wz; I.wx[k] = wx;
            if (split) {
                const size_t SX = I.SX;
                float h, l;
                split_ff(wz, h, l);
                I.ffw[k] = h; I.ffw[SX + k] = l;
                split_ff(wx, h, l);
                I.ffw[2 * SX + k] = h; I.ffw[3 * SX + k] = l;
            }
        } else {
            int j = k - I.SX;
            I.sigu[j] = sgu + sgl; I.wzu[j] = wz; I.wxu[j] = wx;
        }
    }
    const double v[2] = {__longlong_as_double(rpmax), sz};
    constexpr int slot[2] = {0, 1}, kind[2] = {kMaxNonneg, kSum};
    put_parts<2>(I, v, slot, kind, stage);
}

// r_d = H u + h + Gamma'(z1 - z2) + z3 - z4 (Eq. 5a with lambda = z) and the
// predictor right-hand side b = -r_d + J' w (Eq. 7, read with J' r2, see
// the design notes).  One warp per input row; H column j = row j (symmetric).
// Partial: slot 2 max|r_d|.
__global__ void k_rd(const Inst* __restrict__ insts) {
    pdl_wait();
    __shared__ long long ext[32];
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done) return;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    long long rdmax = 0;   // bits of max |r_d|
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < I.n; j += gridDim.x * wpb) {
        const double* hc = I.H64 + (size_t)j * I.n;
        double acc = 0.0;
        for (int k = lane; k < I.n; k += 32) acc += hc[k] * I.u[k];
        acc = warp_sum(acc);
        if (lane == 0) {
            double rd = acc + I.h[j] + I.gz[j] + I.wzu[j];
            I.rd[j] = rd;
            I.b[j] = -rd + I.gw[j] + I.wxu[j];
            const long long a = abs_bits(rd);
            rdmax = a > rdmax ? a : rdmax;
        }
    }
    double v = block_ext<true>(rdmax, ext); put_part(I, 2, v);
}

// Stop test and trace.  nb1: partial count of k_resid, nb2: of k_rd.
__global__ void k_check(const Inst* __restrict__ insts, int nb1, int nb2, int trace_on) {
    pdl_wait();
    __shared__ double fin[3];
    const Inst& I = insts[blockIdx.y];
    Scal* S = I.sc;
    if (S->done) return;
    {
        constexpr int slot[3] = {0, 1, 2}, kind[3] = {kMaxNonneg, kSum, kMaxNonneg};
        const int cnt[3] = {nb1, nb1, nb2};
        reduce_parts<3>(I, slot, kind, cnt, fin);
    }
    const double rp = fin[0], sz = fin[1], rd = fin[2];
    if (threadIdx.x == 0) {
        double mu = S->m > 0 ? sz / S->m : 0.0;
        double res_d = rd / (1.0 + S->hnorm);
        double res_p = rp / (1.0 + S->dnorm);
        double res = fmax(fmax(res_d, res_p), mu);
        S->mu = mu; S->res_d = res_d; S->res_p = res_p; S->res = res;
        if (trace_on && S->iter <= S->max_iter) {
            double* t = I.trace + (size_t)S->iter * kTraceW;
            t[0] = mu; t[1] = res_d; t[2] = res_p; t[3] = 0; t[4] = 0; t[5] = 0; t[6] = 0; t[7] = -1;
        }
        S->refine_iter = 0;
        // a NaN in any row reaches its maximum (the integer order keeps it)
        if (!(res == res) || !(res_d == res_d) || !(res_p == res_p) || !(mu == mu)) { S->done = 1; S->status = 6; }
        else if (res <= S->tol) { S->done = 1; S->status = 0; }
        else if (S->iter >= S->max_iter) { S->done = 1; S->status = 4; }
    }
}

// ---------------------------------------------------------------------------
// Affine (predictor) step: ds = -r_p - J du, dz = -z - Sigma ds per family.
// Stored in ds*/dz*.  Partials: slot 3 largest step to the boundary,
// slot 4 sum(s dz + z ds), slot 5 sum(ds dz) -- so that
// mu_aff = (sum s z + a S4 + a^2 S5)/m in closed form.
// ---------------------------------------------------------------------------

// The largest step to the boundary, min over dv < 0 of v / (-dv), kept as a
// fraction (num, den) with den > 0 and compared by cross-multiplication
// (v * den < num * (-dv)): one FP64 division per thread at the end instead of
// one per candidate (this part's FP64 division costs several FMA-pipe passes).
// The sign test reads the sign bit (integer pipe): a -0 or a negative NaN
// passes it but never wins the cross-multiplied comparison (v > 0).
struct StepMin {
    double num = INFINITY, den = 1.0;
    __device__ __forceinline__ void add(double v, double dv) {
        if (__double_as_longlong(dv) < 0 && v * den < num * -dv) { num = v; den = -dv; }
    }
    __device__ __forceinline__ double value() const { return num / den; }
};

__global__ void k_aff(const Inst* __restrict__ insts) {
    pdl_wait();
    __shared__ double stage[3 * kEwMaxThreads];
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done) return;
    const int total = I.SX + I.n;
    StepMin am;
    double s4 = 0.0, s5 = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        RowView r = row_view(I, k);
        double d = k < I.SX ? I.dxs[k] : I.du[k - I.SX];   // the predictor's solve: du, Gamma du
        double su = *r.s_u, zu = *r.z_u, sl = *r.s_l, zl = *r.z_l;
        double dsu = 0, dzu = 0, dsl = 0, dzl = 0;
        if (r.fu) {
            dsu = -I.rpu[k] - d; dzu = -zu - I.sgu[k] * dsu;
            am.add(su, dsu); am.add(zu, dzu);
            s4 += su * dzu + zu * dsu; s5 += dsu * dzu;
        }
        if (r.fl) {
            dsl = -I.rpl[k] + d; dzl = -zl - I.sgl[k] * dsl;
            am.add(sl, dsl); am.add(zl, dzl);
            s4 += sl * dzl + zl * dsl; s5 += dsl * dzl;
        }
        *r.ds_u = dsu; *r.dz_u = dzu; *r.ds_l = dsl; *r.dz_l = dzl;
    }
    const double v[3] = {am.value(), s4, s5};
    constexpr int slot[3] = {3, 4, 5}, kind[3] = {kMinNonneg, kSum, kSum};
    put_parts<3>(I, v, slot, kind, stage);
    if (!last_arrival(I.sc)) return;
    // The instance's last CTA: alpha_aff = min(1, max step); mu_aff = (sum
    // s z + a S4 + a^2 S5) / m; sigma = (mu_aff/mu)^3 (Mehrotra).  Slot 1
    // (sum s.z) is k_resid's, launched on the same grid.
    __shared__ double fin[4];
    {
        const int nb = gridDim.x;
        constexpr int fslot[4] = {3, 1, 4, 5}, fkind[4] = {kMinNonneg, kSum, kSum, kSum};
        const int cnt[4] = {nb, nb, nb, nb};
        reduce_parts<4>(I, fslot, fkind, cnt, fin);
    }
    if (threadIdx.x == 0) {
        Scal* S = I.sc;
        const double al = fmin(1.0, fin[0]);
        const double mu_aff = S->m > 0 ? (fin[1] + al * fin[2] + al * al * fin[3]) / S->m : 0.0;
        const double ratio_ = S->mu > 0.0 ? mu_aff / S->mu : 0.0;
        S->alpha_aff = al; S->mu_aff = mu_aff;
        S->sigma = ratio_ * ratio_ * ratio_;
    }
}

// Corrector: r_c = s.z + ds_aff.dz_aff - sigma mu (kept in rcu / rcl for
// the step); w = (r_c - z r_p)/s per family, with the iteration's r_p and
// 1/s; wx = w1 - w2 (state rows), wxu = w3 - w4 (input rows).  With split,
// also the float-float split of wx (hi0, lo0 in ffw).
__global__ void k_corr(const Inst* __restrict__ insts, int split) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done) return;
    const double smu = I.sc->sigma * I.sc->mu;
    const int total = I.SX + I.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        RowView r = row_view(I, k);
        double su = *r.s_u, zu = *r.z_u, sl = *r.s_l, zl = *r.z_l;
        double wu = 0, wl = 0;
        if (r.fu) {
            const double rc = su * zu + (*r.ds_u) * (*r.dz_u) - smu;
            I.rcu[k] = rc;
            wu = (rc - zu * I.rpu[k]) * I.rsu[k];
        }
        if (r.fl) {
            const double rc = sl * zl + (*r.ds_l) * (*r.dz_l) - smu;
            I.rcl[k] = rc;
            wl = (rc - zl * I.rpl[k]) * I.rsl[k];
        }
        if (k < I.SX) {
            I.wx[k] = wu - wl;
            if (split) {
                float h, l;
                split_ff(wu - wl, h, l);
                I.ffw[k] = h; I.ffw[(size_t)I.SX + k] = l;
            }
        } else {
            I.wxu[k - I.SX] = wu - wl;
        }
    }
}

// b = -r_d + Gamma' wx + wxu
__global__ void k_rhs(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done) return;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < I.n; j += gridDim.x * blockDim.x)
        I.b[j] = -I.rd[j] + I.gw[j] + I.wxu[j];
}

// Corrector step: ds = -r_p - J du, dz = -(r_c + z ds)/s, with the
// iteration's r_p and 1/s and the corrector's r_c.  Overwrites ds*/dz*.
// Partial: slot 3 max step.  This and the update (k_update) skip an instance
// whose KKT solve of the iteration failed unseen (Scal::spec_fail): the
// iterate stays as it was and the host repeats the iteration.
__global__ void k_step(const Inst* __restrict__ insts, int trace_on) {
    pdl_wait();
    __shared__ double stage[kEwMaxThreads];
    const Inst& I = insts[blockIdx.y];
    if (I.sc->done || I.sc->spec_fail) return;
    const int total = I.SX + I.n;
    StepMin am;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        RowView r = row_view(I, k);
        double d = k < I.SX ? I.dxs[k] : I.du[k - I.SX];   // the corrector's solve: du, Gamma du
        double su = *r.s_u, zu = *r.z_u, sl = *r.s_l, zl = *r.z_l;
        double dsu = 0, dzu = 0, dsl = 0, dzl = 0;
        if (r.fu) {
            dsu = -I.rpu[k] - d; dzu = -(I.rcu[k] + zu * dsu) * I.rsu[k];
            am.add(su, dsu); am.add(zu, dzu);
        }
        if (r.fl) {
            dsl = -I.rpl[k] + d; dzl = -(I.rcl[k] + zl * dsl) * I.rsl[k];
            am.add(sl, dsl); am.add(zl, dzl);
        }
        *r.ds_u = dsu; *r.dz_u = dzu; *r.ds_l = dsl; *r.dz_l = dzl;
    }
    const double v[1] = {am.value()};
    constexpr int slot[1] = {3}, kind[1] = {kMinNonneg};
    put_parts<1>(I, v, slot, kind, stage);
    if (!last_arrival(I.sc)) return;
    // The instance's last CTA: alpha = min(1, tau * max step); the trace row;
    // the iteration count (k_update reads alpha only).
    __shared__ double fin[1];
    {
        constexpr int fslot[1] = {3}, fkind[1] = {kMinNonneg};
        const int cnt[1] = {(int)gridDim.x};
        reduce_parts<1>(I, fslot, fkind, cnt, fin);
    }
    if (threadIdx.x == 0) {
        Scal* S = I.sc;
        const double al = fmin(1.0, S->tau * fin[0]);
        S->alpha = al;
        if (trace_on && S->iter <= S->max_iter) {
            double* t = I.trace + (size_t)S->iter * kTraceW;
            t[3] = S->alpha_aff; t[4] = S->sigma; t[5] = al;
            t[6] = S->refine_iter; t[7] = S->prec_cur;
        }
        S->iter += 1;
    }
}

// One step length for every variable (u, x, s, z).
__global__ void k_update(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    const Scal* S = I.sc;
    if (S->done || S->spec_fail) return;
    const double al = S->alpha;
    const int total = I.SX + I.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        RowView r = row_view(I, k);
        if (k < I.SX) I.x[k] += al * I.dxs[k];
        else I.u[k - I.SX] += al * I.du[k - I.SX];
        *r.s_u += al * (*r.ds_u); *r.z_u += al * (*r.dz_u);
        *r.s_l += al * (*r.ds_l); *r.z_l += al * (*r.dz_l);
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static int ew_blocks(int total_max, int threads) {
    int b = (total_max + threads - 1) / threads;
    return b < 1 ? 1 : (b > kMaxParts ? kMaxParts : b);
}

int device_sm_count() {
    static const int n = []() {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
            v = 1;
        return v;
    }();
    return n;
}

// Grid of the per-row kernels of an iteration (k_resid, k_aff, k_corr,
// k_step, k_update; k_aff's finish reads k_resid's partials, so they share
// it).  Their time is the FP64 work of the most loaded SM: a single instance
// of up to 1024 rows per SM takes one CTA per SM with an equal share of the
// rows (a multiple of 32 threads).  Larger instances and batches keep
// 256-thread CTAs over a grid stride, whose many CTAs spread by themselves
// (1024-thread CTAs of 56 registers would fit one per SM, in ragged waves).
struct EwGrid {
    int nb, threads;
};
static EwGrid ew_grid(int count, int max_total) {
    if (count == 1) {
        const int sms = device_sm_count();
        int th = ((max_total + sms - 1) / sms + 31) / 32 * 32;
        th = th < 64 ? 64 : th;
        if (th <= kEwMaxThreads) return {ew_blocks(max_total, th), th};
    }
    return {ew_blocks(max_total, 256), 256};
}

void launch_init_point(const Inst* d_insts, int count, int max_total, int max_n, double tol,
                       double tau, int max_iter, double refine_tol, int prec, cudaStream_t st, double mu0,
                       double smin) {
    int nb = ew_blocks(max_total, 256);
    LQ_LAUNCH(lq_pdl(k_init_slacks, dim3(nb, count), 256, 0, st, d_insts, mu0, smin));
    LQ_LAUNCH(lq_pdl(k_init_fin, dim3(1, count), 256, 0, st, d_insts, nb, tol, tau, max_iter, refine_tol, prec));
}

void launch_set_u0(const Inst* d_insts, int count, int max_n, cudaStream_t st, int warm) {
    LQ_LAUNCH(lq_pdl(k_set_u0, dim3(ew_blocks(max_n, 256), count), 256, 0, st, d_insts, warm));
}

void launch_resid_check(const Inst* d_insts, int count, int max_total, int max_n, int trace_on,
                        cudaStream_t st, bool do_resid, bool do_rd, int rd_parts, bool split_w) {
    const EwGrid g = ew_grid(count, max_total);
    const int nb1 = g.nb;
    if (do_resid) LQ_LAUNCH(lq_pdl(k_resid, dim3(nb1, count), g.threads, 0, st, d_insts, split_w ? 1 : 0));
    int wpb = 8;
    int nb2 = (max_n + wpb - 1) / wpb;
    nb2 = nb2 > kMaxParts ? kMaxParts : nb2;
    if (do_rd) {
        if (rd_parts & 1) LQ_LAUNCH(lq_pdl(k_rd, dim3(nb2, count), wpb * 32, 0, st, d_insts));
        if (rd_parts & 2) LQ_LAUNCH(lq_pdl(k_check, dim3(1, count), 256, 0, st, d_insts, nb1, nb2, trace_on));
    }
}

void launch_aff(const Inst* d_insts, int count, int max_total, cudaStream_t st) {
    const EwGrid g = ew_grid(count, max_total);
    LQ_LAUNCH(lq_pdl(k_aff, dim3(g.nb, count), g.threads, 0, st, d_insts));
}

void launch_corr(const Inst* d_insts, int count, int max_total, cudaStream_t st, bool split_w) {
    const EwGrid g = ew_grid(count, max_total);
    LQ_LAUNCH(lq_pdl(k_corr, dim3(g.nb, count), g.threads, 0, st, d_insts, split_w ? 1 : 0));
}

void launch_rhs(const Inst* d_insts, int count, int max_n, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_rhs, dim3(ew_blocks(max_n, 256), count), 256, 0, st, d_insts));
}

void launch_step_update(const Inst* d_insts, int count, int max_total, int trace_on,
                        cudaStream_t st) {
    const EwGrid g = ew_grid(count, max_total);
    LQ_LAUNCH(lq_pdl(k_step, dim3(g.nb, count), g.threads, 0, st, d_insts, trace_on));
    LQ_LAUNCH(lq_pdl(k_update, dim3(g.nb, count), g.threads, 0, st, d_insts));
}

}  // namespace lqmpc
