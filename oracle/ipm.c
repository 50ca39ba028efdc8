/*
 * Oracle: plain FP64 CPU interior-point solver for box-constrained LQ-MPC.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant with the
 * CUDA path.
 *
 * What it computes.  The problem is Eq. 1 of the paper:
 *     min  1/2 sum_{t=1}^{N-1} x_t' Q x_t + 1/2 x_N' Qf x_N + 1/2 sum_{t=0}^{N-1} u_t' R u_t
 *          + sum_{t=0}^{N-1} x_t' S u_t
 *     s.t. x_0 = xbar,  x_{t+1} = A x_t + B u_t + w_t,
 *          gl <= E x_t + F u_t <= gu (t = 0..N-1),
 *          xl <= x_t <= xu (t = 1..N),  ul <= u_t <= uu (t = 0..N-1),
 * with S, w and the nc general constraints optional (absent: zero).
 * The bounds on x_0 are dropped because x_0 is fixed (Eq. 1e lists t = 0..T;
 * a fixed x_0 makes them constants).  The 1/2 follows Eq. 3a (Eq. 1a has none;
 * scaling does not move the minimiser).
 *
 * Algorithm.  Mehrotra's predictor-corrector primal-dual method applied to
 * the UNCONDENSED problem in (x, u, lambda, s, z) (Section III poses the
 * barrier problem, Eq. 4, its KKT conditions, Eq. 5, and the Newton system,
 * Eq. 6; here the same Newton system is written before the states are
 * eliminated).  After s and z are eliminated the Newton system is an
 * equality-constrained LQ problem with stage Hessians Q + Sigma_x and
 * R + Sigma_u, solved by a backward Riccati recursion and a forward rollout
 * (the "Riccati-like recursions" the paper names in Section I as the
 * classical sparse alternative).  One step length is applied to every
 * variable (the paper's Algorithm 1 steps v, s, lambda together; with lambda
 * identified with z as Eq. 5b states at the solution, z takes the same step).
 *
 * Readings where the paper is silent (listed again in the design notes):
 *  - initial point: u0 = box midpoint, x0 = rollout, s0 = max(slack, 1),
 *    z0 = 1, lambda0 from the adjoint recursion (zero state-stationarity);
 *  - warm start (not in the paper; the learned warm start starts from a
 *    guess): u0 = the guess moved inside the input box by 1% of the range,
 *    s0 = max(slack, 1e-2), z0 = mu0 / s0, lambda0 as above;
 *  - Mehrotra sigma = (mu_aff / mu)^3, fraction to boundary tau = 0.995;
 *  - stop when max(||r_d||/(1+||h||), ||r_p||/(1+||d||), mu) <= tol, with
 *    h = Gamma' Qbar Phi xbar and d the condensed constraint right-hand side
 *    (Eq. 3b), both computed here from their definitions by rollouts.
 *
 * Sparse storage of A, Q, Qf (CSR) is a representation choice only; every
 * product is the plain sum over the stored nonzeros.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const orc_problem* pb;
    int ns, nu, N, n;
    int m;                      /* number of finite one-sided constraints */
    unsigned char *f1, *f2;     /* finite masks: xu, xl (per state) */
    unsigned char *f3, *f4;     /* finite masks: uu, ul (per input) */
    int nc;                     /* general constraints per stage */
    unsigned char *f5, *f6;     /* finite masks: gu, gl (per constraint row) */
} ctx_t;

/* out = E x + F u (nc rows; x may be NULL for x = 0) */
static void cons_eval(const ctx_t* c, const double* x, const double* u, double* out) {
    const orc_problem* pb = c->pb;
    for (int r = 0; r < c->nc; ++r) {
        double v = 0.0;
        if (x)
            for (int i = 0; i < c->ns; ++i) v += pb->E[r + (size_t)i * c->nc] * x[i];
        for (int a = 0; a < c->nu; ++a) v += pb->F[r + (size_t)a * c->nc] * u[a];
        out[r] = v;
    }
}

/* xo += E' v (if xo), uo += F' v (if uo) */
static void cons_tadd(const ctx_t* c, const double* v, double* xo, double* uo) {
    const orc_problem* pb = c->pb;
    for (int r = 0; r < c->nc; ++r) {
        const double vr = v[r];
        if (vr == 0.0) continue;
        if (xo)
            for (int i = 0; i < c->ns; ++i) xo[i] += pb->E[r + (size_t)i * c->nc] * vr;
        if (uo)
            for (int a = 0; a < c->nu; ++a) uo[a] += pb->F[r + (size_t)a * c->nc] * vr;
    }
}

/* y += alpha * A x  (CSR) */
static void csr_mv_add(int rows, const int* ptr, const int* idx, const double* val,
                       const double* x, double alpha, double* y) {
    for (int r = 0; r < rows; ++r) {
        double acc = 0.0;
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) acc += val[k] * x[idx[k]];
        y[r] += alpha * acc;
    }
}

/* y += alpha * A' x  (CSR) */
static void csr_mtv_add(int rows, const int* ptr, const int* idx, const double* val,
                        const double* x, double alpha, double* y) {
    for (int r = 0; r < rows; ++r) {
        double xr = alpha * x[r];
        if (xr == 0.0) continue;
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) y[idx[k]] += val[k] * xr;
    }
}

static double mid_of_box(double lo, double hi) {
    int fl = isfinite(lo), fh = isfinite(hi);
    if (fl && fh) return 0.5 * (lo + hi);
    if (fl) return lo + 1.0;
    if (fh) return hi - 1.0;
    return 0.0;
}

/* x[0] = xbar; x[t+1] = A x[t] + B u[t] + w[t] */
static void rollout(const ctx_t* c, const double* xbar, const double* u, double* x) {
    const orc_problem* pb = c->pb;
    int ns = c->ns, nu = c->nu;
    memcpy(x, xbar, sizeof(double) * ns);
    for (int t = 0; t < c->N; ++t) {
        double* xn = x + (size_t)(t + 1) * ns;
        if (pb->w) memcpy(xn, pb->w + (size_t)t * ns, sizeof(double) * ns);
        else memset(xn, 0, sizeof(double) * ns);
        csr_mv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, x + (size_t)t * ns, 1.0, xn);
        for (int j = 0; j < nu; ++j) {
            double uj = u[t * nu + j];
            if (uj == 0.0) continue;
            const double* bj = pb->B + (size_t)j * ns;
            for (int i = 0; i < ns; ++i) xn[i] += bj[i] * uj;
        }
    }
}

/* Dense Cholesky of an n x n column-major SPD matrix in place (lower).
 * Returns 0 on success, k+1 if the k-th pivot is not positive. */
static int chol_small(int n, double* a) {
    for (int j = 0; j < n; ++j) {
        double d = a[j + j * n];
        for (int k = 0; k < j; ++k) d -= a[j + k * n] * a[j + k * n];
        if (!(d > 0.0)) return j + 1;
        d = sqrt(d);
        a[j + j * n] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = a[i + j * n];
            for (int k = 0; k < j; ++k) v -= a[i + k * n] * a[j + k * n];
            a[i + j * n] = v / d;
        }
    }
    return 0;
}

/* Solve (L L') x = b in place, L lower n x n column-major. */
static void chol_solve_small(int n, const double* L, double* b) {
    for (int i = 0; i < n; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[i + k * n] * b[k];
        b[i] = v / L[i + i * n];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < n; ++k) v -= L[k + i * n] * b[k];
        b[i] = v / L[i + i * n];
    }
}

/* Per-iteration factorisation of the Riccati recursion. */
typedef struct {
    double* bpat;   /* N stages: ns x nu, (B' P_{t+1} A)' stored column-major */
    double* hchol;  /* N stages: nu x nu Cholesky of R + Sigma_u + B' P_{t+1} B */
    double* pe;     /* N stages: P_{t+1} e_t (affine dynamics term) */
    double *P, *Pn, *PA, *PB, *Y;
} fact_t;

/*
 * Backward Riccati sweep: P_N = Qf + diag(Sigma_x,N);
 * for t = N-1..0:  Hhat_t = R + diag(Sigma_u,t) + F' Sigma_c,t F + B' P_{t+1} B,
 *                  K'_t = A' P_{t+1} B + S + E' Sigma_c,t F     (bpat, ns x nu)
 *                  P_t = Q + diag(Sigma_x,t) + E' Sigma_c,t E + A' P_{t+1} A
 *                        - K'_t Hhat_t^{-1} K'_t'              (t >= 1).
 * Sigma_c,t (sigc, nc per stage) weighs stage t's general constraint rows.
 * e_t is the dynamics residual (zero for a dynamics-feasible iterate).
 */
static int riccati_factor(const ctx_t* c, const double* sigx, const double* sigu,
                          const double* sigc, const double* e, fact_t* f) {
    const orc_problem* pb = c->pb;
    int ns = c->ns, nu = c->nu, N = c->N;
    size_t nn = (size_t)ns * ns;
    double* Pn = f->Pn;   /* P_{t+1} */
    double* Pt = f->P;    /* P_t */
    /* P_N = Qf + diag(sigx_N) */
    memset(Pn, 0, sizeof(double) * nn);
    for (int r = 0; r < ns; ++r)
        for (int k = pb->qf_ptr[r]; k < pb->qf_ptr[r + 1]; ++k)
            Pn[r + (size_t)pb->qf_idx[k] * ns] += pb->qf_val[k];
    for (int i = 0; i < ns; ++i) Pn[i + (size_t)i * ns] += sigx[(size_t)(N - 1) * ns + i];

    for (int t = N - 1; t >= 0; --t) {
        double* bpat = f->bpat + (size_t)t * ns * nu;
        double* hc = f->hchol + (size_t)t * nu * nu;
        double* pe = f->pe + (size_t)t * ns;
        /* PB = P_{t+1} B */
        memset(f->PB, 0, sizeof(double) * ns * nu);
        for (int j = 0; j < nu; ++j) {
            const double* bj = pb->B + (size_t)j * ns;
            double* out = f->PB + (size_t)j * ns;
            for (int k = 0; k < ns; ++k) {
                double b = bj[k];
                if (b == 0.0) continue;
                const double* pk = Pn + (size_t)k * ns;
                for (int i = 0; i < ns; ++i) out[i] += pk[i] * b;
            }
        }
        /* Hhat = R + diag(sigu_t) + B' PB */
        for (int a = 0; a < nu; ++a)
            for (int b = 0; b < nu; ++b) {
                double v = pb->R[a + b * nu];
                const double* ba = pb->B + (size_t)a * ns;
                const double* pbb = f->PB + (size_t)b * ns;
                for (int k = 0; k < ns; ++k) v += ba[k] * pbb[k];
                hc[a + b * nu] = v;
            }
        for (int a = 0; a < nu; ++a) hc[a + a * nu] += sigu[t * nu + a];
        const double* sc = c->nc ? sigc + (size_t)t * c->nc : NULL;
        for (int r = 0; sc && r < c->nc; ++r)          /* F' Sigma_c F */
            for (int a = 0; a < nu; ++a)
                for (int b = 0; b < nu; ++b)
                    hc[a + b * nu] += pb->F[r + (size_t)a * c->nc] * sc[r] * pb->F[r + (size_t)b * c->nc];
        if (chol_small(nu, hc)) return ORC_ERR_NOT_PD;
        /* bpat[:, c] = ((PB)' A)' [:, c] = A' PB[:, c] */
        memset(bpat, 0, sizeof(double) * ns * nu);
        for (int j = 0; j < nu; ++j)
            csr_mtv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, f->PB + (size_t)j * ns, 1.0,
                        bpat + (size_t)j * ns);
        if (pb->S)                                      /* cross term S */
            for (size_t k = 0; k < (size_t)ns * nu; ++k) bpat[k] += pb->S[k];
        for (int r = 0; sc && r < c->nc; ++r)          /* E' Sigma_c F */
            for (int a = 0; a < nu; ++a) {
                const double fa = sc[r] * pb->F[r + (size_t)a * c->nc];
                if (fa == 0.0) continue;
                for (int i = 0; i < ns; ++i) bpat[i + (size_t)a * ns] += pb->E[r + (size_t)i * c->nc] * fa;
            }
        /* pe = P_{t+1} e_t */
        const double* et = e + (size_t)t * ns;
        memset(pe, 0, sizeof(double) * ns);
        for (int k = 0; k < ns; ++k) {
            double ek = et[k];
            if (ek == 0.0) continue;
            const double* pk = Pn + (size_t)k * ns;
            for (int i = 0; i < ns; ++i) pe[i] += pk[i] * ek;
        }
        if (t == 0) break;
        /* PA = P_{t+1} A : PA[:, j] += a_kj P[:, k] */
        memset(f->PA, 0, sizeof(double) * nn);
        for (int k = 0; k < ns; ++k) {
            const double* pk = Pn + (size_t)k * ns;
            for (int q = pb->a_ptr[k]; q < pb->a_ptr[k + 1]; ++q) {
                double a = pb->a_val[q];
                double* out = f->PA + (size_t)pb->a_idx[q] * ns;
                for (int i = 0; i < ns; ++i) out[i] += a * pk[i];
            }
        }
        /* P_t = A' PA + Q + diag(sigx_t) - bpat Hhat^{-1} bpat' */
        memset(Pt, 0, sizeof(double) * nn);
        for (int j = 0; j < ns; ++j)
            csr_mtv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, f->PA + (size_t)j * ns, 1.0,
                        Pt + (size_t)j * ns);
        for (int r = 0; r < ns; ++r)
            for (int k = pb->q_ptr[r]; k < pb->q_ptr[r + 1]; ++k)
                Pt[r + (size_t)pb->q_idx[k] * ns] += pb->q_val[k];
        for (int i = 0; i < ns; ++i) Pt[i + (size_t)i * ns] += sigx[(size_t)(t - 1) * ns + i];
        for (int r = 0; sc && r < c->nc; ++r) {        /* E' Sigma_c E */
            if (sc[r] == 0.0) continue;
            for (int j = 0; j < ns; ++j) {
                const double ej = sc[r] * pb->E[r + (size_t)j * c->nc];
                if (ej == 0.0) continue;
                for (int i = 0; i < ns; ++i) Pt[i + (size_t)j * ns] += pb->E[r + (size_t)i * c->nc] * ej;
            }
        }
        /* Y = Hhat^{-1} bpat'  (nu x ns), column j = Hhat^{-1} bpat[j, :]' */
        for (int j = 0; j < ns; ++j) {
            double* yj = f->Y + (size_t)j * nu;
            for (int a = 0; a < nu; ++a) yj[a] = bpat[j + (size_t)a * ns];
            chol_solve_small(nu, hc, yj);
        }
        for (int j = 0; j < ns; ++j) {
            double* pj = Pt + (size_t)j * ns;
            const double* yj = f->Y + (size_t)j * nu;
            for (int a = 0; a < nu; ++a) {
                double y = yj[a];
                const double* ba = bpat + (size_t)a * ns;
                for (int i = 0; i < ns; ++i) pj[i] -= ba[i] * y;
            }
        }
        /* symmetrise */
        for (int j = 0; j < ns; ++j)
            for (int i = j + 1; i < ns; ++i) {
                double v = 0.5 * (Pt[i + (size_t)j * ns] + Pt[j + (size_t)i * ns]);
                Pt[i + (size_t)j * ns] = v;
                Pt[j + (size_t)i * ns] = v;
            }
        double* tmp = Pn; Pn = Pt; Pt = tmp;
    }
    return 0;
}

/*
 * Solve the LQ Newton subproblem with linear terms q (states t=1..N, stored
 * at (t-1)*ns) and r (inputs), dynamics offset e:
 *   backward: p_N = q_N; phat = p_{t+1} + P_{t+1} e_t; g_t = r_t + B' phat;
 *             k_t = -Hhat^{-1} g_t; p_t = q_t + A' phat + bpat k_t;
 *   forward:  dx_0 = 0; du_t = -Hhat^{-1}(bpat' dx_t) + k_t;
 *             dx_{t+1} = A dx_t + B du_t + e_t.
 * dx is (N+1)*ns with dx_0 = 0.
 */
static void riccati_solve(const ctx_t* c, const fact_t* f, const double* q, const double* r,
                          const double* e, double* dx, double* du, double* work) {
    const orc_problem* pb = c->pb;
    int ns = c->ns, nu = c->nu, N = c->N;
    double* p = work;            /* ns */
    double* ph = work + ns;      /* ns */
    double* g = work + 2 * ns;   /* nu */
    double* kk = work + 2 * ns + nu;   /* N*nu */
    memcpy(p, q + (size_t)(N - 1) * ns, sizeof(double) * ns);
    for (int t = N - 1; t >= 0; --t) {
        const double* bpat = f->bpat + (size_t)t * ns * nu;
        const double* hc = f->hchol + (size_t)t * nu * nu;
        const double* pe = f->pe + (size_t)t * ns;
        for (int i = 0; i < ns; ++i) ph[i] = p[i] + pe[i];
        for (int a = 0; a < nu; ++a) {
            double v = r[t * nu + a];
            const double* ba = pb->B + (size_t)a * ns;
            for (int i = 0; i < ns; ++i) v += ba[i] * ph[i];
            g[a] = v;
        }
        chol_solve_small(nu, hc, g);
        double* kt = kk + (size_t)t * nu;
        for (int a = 0; a < nu; ++a) kt[a] = -g[a];
        if (t == 0) break;
        const double* qt = q + (size_t)(t - 1) * ns;
        for (int i = 0; i < ns; ++i) p[i] = qt[i];
        csr_mtv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, ph, 1.0, p);
        for (int a = 0; a < nu; ++a) {
            const double* ba = bpat + (size_t)a * ns;
            double ka = kt[a];
            for (int i = 0; i < ns; ++i) p[i] += ba[i] * ka;
        }
    }
    memset(dx, 0, sizeof(double) * ns);
    for (int t = 0; t < N; ++t) {
        const double* bpat = f->bpat + (size_t)t * ns * nu;
        const double* hc = f->hchol + (size_t)t * nu * nu;
        const double* xt = dx + (size_t)t * ns;
        for (int a = 0; a < nu; ++a) {
            const double* ba = bpat + (size_t)a * ns;
            double v = 0.0;
            for (int i = 0; i < ns; ++i) v += ba[i] * xt[i];
            g[a] = v;
        }
        chol_solve_small(nu, hc, g);
        for (int a = 0; a < nu; ++a) du[t * nu + a] = -g[a] + kk[(size_t)t * nu + a];
        double* xn = dx + (size_t)(t + 1) * ns;
        memcpy(xn, e + (size_t)t * ns, sizeof(double) * ns);
        csr_mv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, xt, 1.0, xn);
        for (int a = 0; a < nu; ++a) {
            double ua = du[t * nu + a];
            const double* ba = pb->B + (size_t)a * ns;
            for (int i = 0; i < ns; ++i) xn[i] += ba[i] * ua;
        }
    }
}

/* Adjoint recursion: lam_N = Qt_N dx_N + q_N; lam_t = Qt_t dx_t + q_t + A' lam_{t+1}.
 * Qt_t = Q (Qf at N) + diag(sigx_t).  lam has (N+1)*ns entries, lam_0 unused. */
static void adjoint(const ctx_t* c, const double* dx, const double* q, const double* sigx,
                    double* lam) {
    const orc_problem* pb = c->pb;
    int ns = c->ns, N = c->N;
    for (int t = N; t >= 1; --t) {
        double* lt = lam + (size_t)t * ns;
        const double* xt = dx + (size_t)t * ns;
        for (int i = 0; i < ns; ++i)
            lt[i] = q[(size_t)(t - 1) * ns + i] + (sigx ? sigx[(size_t)(t - 1) * ns + i] * xt[i] : 0.0);
        if (t == N) csr_mv_add(ns, pb->qf_ptr, pb->qf_idx, pb->qf_val, xt, 1.0, lt);
        else {
            csr_mv_add(ns, pb->q_ptr, pb->q_idx, pb->q_val, xt, 1.0, lt);
            csr_mtv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, lam + (size_t)(t + 1) * ns, 1.0, lt);
        }
    }
}

/* The stage terms that couple x_t and u_t (t = 1..N-1 for the state rows,
 * t = 0..N-1 for the inputs): qx_t += S u_t + E' (za_t - zb_t) and, when
 * ru and x are given, ru_t += S' x_t + F' (za_t - zb_t) (x_0 = xbar; x holds
 * x_0..x_N).  za, zb: nc per stage (NULL when nc = 0). */
static void stage_terms(const ctx_t* c, const double* u, const double* za, const double* zb, double* qx,
                        double* ru, const double* x) {
    const orc_problem* pb = c->pb;
    const int ns = c->ns, nu = c->nu, N = c->N, nc = c->nc;
    double* dz = nc ? malloc(sizeof(double) * nc) : NULL;
    for (int t = 0; t < N; ++t) {
        double* qt = t >= 1 ? qx + (size_t)(t - 1) * ns : NULL;
        if (pb->S && qt)
            for (int a = 0; a < nu; ++a) {
                const double ua = u[t * nu + a];
                for (int i = 0; i < ns; ++i) qt[i] += pb->S[i + (size_t)a * ns] * ua;
            }
        if (ru && pb->S)
            for (int a = 0; a < nu; ++a) {
                double v = 0.0;
                for (int i = 0; i < ns; ++i) v += pb->S[i + (size_t)a * ns] * x[(size_t)t * ns + i];
                ru[t * nu + a] += v;
            }
        if (nc) {
            for (int r = 0; r < nc; ++r) dz[r] = za[(size_t)t * nc + r] - zb[(size_t)t * nc + r];
            cons_tadd(c, dz, qt, ru ? ru + t * nu : NULL);
        }
    }
    free(dz);
}

static double vmaxabs(const double* v, size_t n) {
    double m = 0.0;
    for (size_t i = 0; i < n; ++i) { double a = fabs(v[i]); if (a > m || a != a) m = a; }
    return m;
}

int orc_ipm_solve(const orc_problem* pb, const double* xbar, const orc_options* op,
                  double* u_out, double* x_out, double* z_out, orc_stats* st, double* trace) {
    ctx_t c;
    c.pb = pb; c.ns = pb->ns; c.nu = pb->nu; c.N = pb->N; c.n = pb->nu * pb->N;
    int ns = c.ns, nu = c.nu, N = c.N, n = c.n;
    size_t SX = (size_t)N * ns;          /* state rows t = 1..N */
    size_t XT = (size_t)(N + 1) * ns;    /* trajectories incl. t = 0 */
    double tol = op ? op->tol : 1e-8;
    int max_iter = op ? op->max_iter : 100;
    double tau = op ? op->tau : 0.995;

    c.f1 = malloc(ns); c.f2 = malloc(ns); c.f3 = malloc(nu); c.f4 = malloc(nu);
    c.m = 0;
    for (int i = 0; i < ns; ++i) {
        c.f1[i] = isfinite(pb->xu[i]) != 0; c.f2[i] = isfinite(pb->xl[i]) != 0;
        c.m += N * (c.f1[i] + c.f2[i]);
    }
    for (int j = 0; j < nu; ++j) {
        c.f3[j] = isfinite(pb->uu[j]) != 0; c.f4[j] = isfinite(pb->ul[j]) != 0;
        c.m += N * (c.f3[j] + c.f4[j]);
    }
    c.nc = (pb->nc > 0 && pb->E && pb->F && pb->gl && pb->gu) ? pb->nc : 0;
    const int nc = c.nc;
    const size_t CX = (size_t)N * nc;   /* general constraint rows, stage t at t*nc */
    c.f5 = malloc(nc + 1); c.f6 = malloc(nc + 1);
    for (int r = 0; r < nc; ++r) {
        c.f5[r] = isfinite(pb->gu[r]) != 0; c.f6[r] = isfinite(pb->gl[r]) != 0;
        c.m += N * (c.f5[r] + c.f6[r]);
    }

    /* variables */
    double* u = calloc(n, sizeof(double));
    double* x = calloc(XT, sizeof(double));
    double* lam = calloc(XT, sizeof(double));
    double *s1 = calloc(SX, 8), *s2 = calloc(SX, 8), *z1 = calloc(SX, 8), *z2 = calloc(SX, 8);
    double *s3 = calloc(n, 8), *s4 = calloc(n, 8), *z3 = calloc(n, 8), *z4 = calloc(n, 8);
    /* residuals and work */
    double *rx = calloc(SX, 8), *ru = calloc(n, 8), *rdyn = calloc(SX, 8);
    double *rp1 = calloc(SX, 8), *rp2 = calloc(SX, 8), *rp3 = calloc(n, 8), *rp4 = calloc(n, 8);
    double *sigx = calloc(SX, 8), *sigu = calloc(n, 8);
    double *q = calloc(SX, 8), *r = calloc(n, 8);
    double *dx = calloc(XT, 8), *du = calloc(n, 8), *dlam = calloc(XT, 8);
    double *ds1 = calloc(SX, 8), *ds2 = calloc(SX, 8), *ds3 = calloc(n, 8), *ds4 = calloc(n, 8);
    double *dz1 = calloc(SX, 8), *dz2 = calloc(SX, 8), *dz3 = calloc(n, 8), *dz4 = calloc(n, 8);
    double *rc1 = calloc(SX, 8), *rc2 = calloc(SX, 8), *rc3 = calloc(n, 8), *rc4 = calloc(n, 8);
    /* general constraints: value c_t = E x_t + F u_t, slacks/duals (upper 5,
     * lower 6), residuals, steps, Sigma_c and the per-stage linear terms */
    double *cv = calloc(CX + 1, 8), *s5 = calloc(CX + 1, 8), *z5 = calloc(CX + 1, 8), *s6 = calloc(CX + 1, 8);
    double *z6 = calloc(CX + 1, 8), *rp5 = calloc(CX + 1, 8), *rp6 = calloc(CX + 1, 8), *rc5 = calloc(CX + 1, 8);
    double *rc6 = calloc(CX + 1, 8), *ds5 = calloc(CX + 1, 8), *dz5 = calloc(CX + 1, 8), *ds6 = calloc(CX + 1, 8);
    double *dz6 = calloc(CX + 1, 8), *sigc = calloc(CX + 1, 8), *wc = calloc(CX + 1, 8), *dcv = calloc(CX + 1, 8);
    double* work = calloc(2 * (size_t)ns + nu + n + 8, 8);
    double* tmp = calloc(XT, 8);
    fact_t f;
    f.bpat = calloc((size_t)N * ns * nu, 8);
    f.hchol = calloc((size_t)N * nu * nu, 8);
    f.pe = calloc((size_t)N * ns, 8);
    f.P = calloc((size_t)ns * ns, 8); f.Pn = calloc((size_t)ns * ns, 8);
    f.PA = calloc((size_t)ns * ns, 8);
    f.PB = calloc((size_t)ns * nu, 8); f.Y = calloc((size_t)ns * nu, 8);

    int status = ORC_OK;
    int it = 0;
    double mu = 0, res_d = 0, res_p = 0, res = 0;

    /* ||h|| and ||d||: h = Gamma' Qbar y, y = rollout with u = 0 (the
     * condensed linear term of Eq. 3a and the right-hand side of Eq. 3b). */
    double hnorm, dnorm = 0.0;
    {
        memset(u, 0, sizeof(double) * n);
        rollout(&c, xbar, u, x);
        memset(q, 0, sizeof(double) * SX);
        adjoint(&c, x, q, NULL, lam);
        double hm = 0.0;
        for (int t = 0; t < N; ++t)
            for (int a = 0; a < nu; ++a) {
                const double* ba = pb->B + (size_t)a * ns;
                const double* lt = lam + (size_t)(t + 1) * ns;
                double v = 0.0;
                for (int i = 0; i < ns; ++i) v += ba[i] * lt[i];
                if (fabs(v) > hm) hm = fabs(v);
            }
        if (pb->S) {                     /* + S' y_t (y_0 = xbar) */
            hm = 0.0;
            for (int t = 0; t < N; ++t)
                for (int a = 0; a < nu; ++a) {
                    const double* ba = pb->B + (size_t)a * ns;
                    const double* lt = lam + (size_t)(t + 1) * ns;
                    const double* sa = pb->S + (size_t)a * ns;
                    const double* yt = x + (size_t)t * ns;
                    double v = 0.0, vs = 0.0;
                    for (int i = 0; i < ns; ++i) v += ba[i] * lt[i];
                    for (int i = 0; i < ns; ++i) vs += sa[i] * yt[i];
                    if (fabs(v + vs) > hm) hm = fabs(v + vs);
                }
        }
        hnorm = hm;
        for (int t = 0; t < N && nc; ++t) {   /* general rows at u = 0: E y_t */
            cons_eval(&c, x + (size_t)t * ns, u, cv);
            for (int r2 = 0; r2 < nc; ++r2) {
                if (c.f5[r2] && fabs(pb->gu[r2] - cv[r2]) > dnorm) dnorm = fabs(pb->gu[r2] - cv[r2]);
                if (c.f6[r2] && fabs(cv[r2] - pb->gl[r2]) > dnorm) dnorm = fabs(cv[r2] - pb->gl[r2]);
            }
        }
        for (int t = 1; t <= N; ++t)
            for (int i = 0; i < ns; ++i) {
                double y = x[(size_t)t * ns + i];
                if (c.f1[i] && fabs(pb->xu[i] - y) > dnorm) dnorm = fabs(pb->xu[i] - y);
                if (c.f2[i] && fabs(y - pb->xl[i]) > dnorm) dnorm = fabs(y - pb->xl[i]);
            }
        for (int j = 0; j < nu; ++j) {
            if (c.f3[j] && fabs(pb->uu[j]) > dnorm) dnorm = fabs(pb->uu[j]);
            if (c.f4[j] && fabs(pb->ul[j]) > dnorm) dnorm = fabs(pb->ul[j]);
        }
    }

    /* initial point.  Cold: u = box midpoints, s = max(slack, 1), z = 1.
     * Warm (u_init given): u = the guess moved inside the box by a margin,
     * s = max(slack, 1e-2), z = mu0 / s (complementarity mu0 on every pair). */
    const double* ui = op ? op->u_init : NULL;
    const double mu0 = (op && op->mu0 > 0.0) ? op->mu0 : 1e-2;
    const double sfl = ui ? 1e-2 : 1.0;
    for (int t = 0; t < N; ++t)
        for (int j = 0; j < nu; ++j) {
            if (!ui) { u[t * nu + j] = mid_of_box(pb->ul[j], pb->uu[j]); continue; }
            double lo = pb->ul[j], hi = pb->uu[j], v = ui[t * nu + j];
            int fl = isfinite(lo), fh = isfinite(hi);
            double margin = (fl && fh) ? 0.01 * (hi - lo) : 0.01;
            if (fl && v < lo + margin) v = lo + margin;
            if (fh && v > hi - margin) v = hi - margin;
            if (fl && fh && hi - lo <= 2.0 * margin) v = 0.5 * (lo + hi);
            u[t * nu + j] = v;
        }
    rollout(&c, xbar, u, x);
#define DUAL0(sv) (ui ? mu0 / (sv) : 1.0)
    for (int t = 1; t <= N; ++t)
        for (int i = 0; i < ns; ++i) {
            size_t k = (size_t)(t - 1) * ns + i;
            double xi = x[(size_t)t * ns + i];
            s1[k] = c.f1[i] ? fmax(pb->xu[i] - xi, sfl) : 1.0; z1[k] = c.f1[i] ? DUAL0(s1[k]) : 0.0;
            s2[k] = c.f2[i] ? fmax(xi - pb->xl[i], sfl) : 1.0; z2[k] = c.f2[i] ? DUAL0(s2[k]) : 0.0;
        }
    for (int t = 0; t < N; ++t)
        for (int j = 0; j < nu; ++j) {
            int k = t * nu + j;
            s3[k] = c.f3[j] ? fmax(pb->uu[j] - u[k], sfl) : 1.0; z3[k] = c.f3[j] ? DUAL0(s3[k]) : 0.0;
            s4[k] = c.f4[j] ? fmax(u[k] - pb->ul[j], sfl) : 1.0; z4[k] = c.f4[j] ? DUAL0(s4[k]) : 0.0;
        }
    for (int t = 0; t < N && nc; ++t) {
        cons_eval(&c, x + (size_t)t * ns, u + (size_t)t * nu, cv + (size_t)t * nc);
        for (int r2 = 0; r2 < nc; ++r2) {
            size_t k = (size_t)t * nc + r2;
            s5[k] = c.f5[r2] ? fmax(pb->gu[r2] - cv[k], sfl) : 1.0; z5[k] = c.f5[r2] ? DUAL0(s5[k]) : 0.0;
            s6[k] = c.f6[r2] ? fmax(cv[k] - pb->gl[r2], sfl) : 1.0; z6[k] = c.f6[r2] ? DUAL0(s6[k]) : 0.0;
        }
    }
#undef DUAL0
    /* lambda0: zero state stationarity, lam_t = Q x_t + z1 - z2 + S u_t
     * + E'(z5 - z6) + A' lam_{t+1} */
    for (size_t k = 0; k < SX; ++k) q[k] = z1[k] - z2[k];
    stage_terms(&c, u, z5, z6, q, NULL, NULL);
    adjoint(&c, x, q, NULL, lam);

    for (it = 0;; ++it) {
        /* --- residuals (Eq. 5) --- */
        /* r_x,t = Q_t x_t - lam_t + A' lam_{t+1} + z1_t - z2_t */
        for (int t = 1; t <= N; ++t) {
            double* rt = rx + (size_t)(t - 1) * ns;
            const double* xt = x + (size_t)t * ns;
            const double* lt = lam + (size_t)t * ns;
            for (int i = 0; i < ns; ++i) {
                size_t k = (size_t)(t - 1) * ns + i;
                rt[i] = -lt[i] + z1[k] - z2[k];
            }
            if (t == N) csr_mv_add(ns, pb->qf_ptr, pb->qf_idx, pb->qf_val, xt, 1.0, rt);
            else {
                csr_mv_add(ns, pb->q_ptr, pb->q_idx, pb->q_val, xt, 1.0, rt);
                csr_mtv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, lam + (size_t)(t + 1) * ns, 1.0, rt);
            }
        }
        /* r_u,t = R u_t + B' lam_{t+1} + z3 - z4 */
        for (int t = 0; t < N; ++t)
            for (int a = 0; a < nu; ++a) {
                double v = 0.0;
                for (int b = 0; b < nu; ++b) v += pb->R[a + b * nu] * u[t * nu + b];
                const double* ba = pb->B + (size_t)a * ns;
                const double* lt = lam + (size_t)(t + 1) * ns;
                for (int i = 0; i < ns; ++i) v += ba[i] * lt[i];
                ru[t * nu + a] = v + z3[t * nu + a] - z4[t * nu + a];
            }
        /* + S u_t + E'(z5 - z6) (states), S' x_t + F'(z5 - z6) (inputs) */
        stage_terms(&c, u, z5, z6, rx, ru, x);
        /* r_dyn,t = A x_t + B u_t + w_t - x_{t+1} */
        for (int t = 0; t < N; ++t) {
            double* rt = rdyn + (size_t)t * ns;
            const double* xt1 = x + (size_t)(t + 1) * ns;
            for (int i = 0; i < ns; ++i) rt[i] = -xt1[i];
            if (pb->w)
                for (int i = 0; i < ns; ++i) rt[i] += pb->w[(size_t)t * ns + i];
            csr_mv_add(ns, pb->a_ptr, pb->a_idx, pb->a_val, x + (size_t)t * ns, 1.0, rt);
            for (int a = 0; a < nu; ++a) {
                double ua = u[t * nu + a];
                const double* ba = pb->B + (size_t)a * ns;
                for (int i = 0; i < ns; ++i) rt[i] += ba[i] * ua;
            }
        }
        /* primal residuals of Jv - d + s = 0 (Eq. 5c), per family */
        double rpmax = vmaxabs(rdyn, SX), sz = 0.0;
        for (int t = 1; t <= N; ++t)
            for (int i = 0; i < ns; ++i) {
                size_t k = (size_t)(t - 1) * ns + i;
                double xi = x[(size_t)t * ns + i];
                rp1[k] = c.f1[i] ? xi + s1[k] - pb->xu[i] : 0.0;
                rp2[k] = c.f2[i] ? -xi + s2[k] + pb->xl[i] : 0.0;
                if (fabs(rp1[k]) > rpmax) rpmax = fabs(rp1[k]);
                if (fabs(rp2[k]) > rpmax) rpmax = fabs(rp2[k]);
                sz += (c.f1[i] ? s1[k] * z1[k] : 0.0) + (c.f2[i] ? s2[k] * z2[k] : 0.0);
            }
        for (int t = 0; t < N; ++t)
            for (int j = 0; j < nu; ++j) {
                int k = t * nu + j;
                rp3[k] = c.f3[j] ? u[k] + s3[k] - pb->uu[j] : 0.0;
                rp4[k] = c.f4[j] ? -u[k] + s4[k] + pb->ul[j] : 0.0;
                if (fabs(rp3[k]) > rpmax) rpmax = fabs(rp3[k]);
                if (fabs(rp4[k]) > rpmax) rpmax = fabs(rp4[k]);
                sz += (c.f3[j] ? s3[k] * z3[k] : 0.0) + (c.f4[j] ? s4[k] * z4[k] : 0.0);
            }
        for (int t = 0; t < N && nc; ++t) {   /* general rows: c_t + s5 - gu, -c_t + s6 + gl */
            cons_eval(&c, x + (size_t)t * ns, u + (size_t)t * nu, cv + (size_t)t * nc);
            for (int r2 = 0; r2 < nc; ++r2) {
                size_t k = (size_t)t * nc + r2;
                rp5[k] = c.f5[r2] ? cv[k] + s5[k] - pb->gu[r2] : 0.0;
                rp6[k] = c.f6[r2] ? -cv[k] + s6[k] + pb->gl[r2] : 0.0;
                if (fabs(rp5[k]) > rpmax) rpmax = fabs(rp5[k]);
                if (fabs(rp6[k]) > rpmax) rpmax = fabs(rp6[k]);
                sz += (c.f5[r2] ? s5[k] * z5[k] : 0.0) + (c.f6[r2] ? s6[k] * z6[k] : 0.0);
            }
        }
        double rdmax = vmaxabs(ru, n);
        double rxm = vmaxabs(rx, SX);
        if (rxm > rdmax || rxm != rxm) rdmax = rxm;
        mu = c.m > 0 ? sz / c.m : 0.0;
        res_d = rdmax / (1.0 + hnorm);
        res_p = rpmax / (1.0 + dnorm);
        res = fmax(fmax(res_d, res_p), mu);
        if (trace && it < max_iter + 1) {
            double* tr = trace + (size_t)it * ORC_TRACE_W;
            tr[0] = mu; tr[1] = res_d; tr[2] = res_p; tr[3] = 0; tr[4] = 0; tr[5] = 0;
        }
        if (!(res == res)) { status = ORC_ERR_NAN; break; }
        if (res <= tol) break;
        if (it >= max_iter) { status = ORC_ERR_MAXITER; break; }

        /* --- Sigma = S^{-1} Z (Eq. 6), per state and input row --- */
        for (size_t k = 0; k < SX; ++k) sigx[k] = z1[k] / s1[k] + z2[k] / s2[k];
        for (int k = 0; k < n; ++k) sigu[k] = z3[k] / s3[k] + z4[k] / s4[k];
        for (size_t k = 0; k < CX; ++k) sigc[k] = z5[k] / s5[k] + z6[k] / s6[k];
        int fs = riccati_factor(&c, sigx, sigu, sigc, rdyn, &f);
        if (fs) { status = fs; break; }

        double alpha_aff = 1.0, sigma = 0.0, alpha = 1.0;
        for (int pass = 0; pass < 2; ++pass) {
            /* complementarity right-hand side: predictor s.z, corrector
             * s.z + ds_aff.dz_aff - sigma mu */
            if (pass == 0) {
                for (size_t k = 0; k < SX; ++k) { rc1[k] = s1[k] * z1[k]; rc2[k] = s2[k] * z2[k]; }
                for (int k = 0; k < n; ++k) { rc3[k] = s3[k] * z3[k]; rc4[k] = s4[k] * z4[k]; }
                for (size_t k = 0; k < CX; ++k) { rc5[k] = s5[k] * z5[k]; rc6[k] = s6[k] * z6[k]; }
            } else {
                double smu = sigma * mu;
                for (int t = 1; t <= N; ++t)
                    for (int i = 0; i < ns; ++i) {
                        size_t k = (size_t)(t - 1) * ns + i;
                        rc1[k] = c.f1[i] ? s1[k] * z1[k] + ds1[k] * dz1[k] - smu : 0.0;
                        rc2[k] = c.f2[i] ? s2[k] * z2[k] + ds2[k] * dz2[k] - smu : 0.0;
                    }
                for (int t = 0; t < N; ++t)
                    for (int j = 0; j < nu; ++j) {
                        int k = t * nu + j;
                        rc3[k] = c.f3[j] ? s3[k] * z3[k] + ds3[k] * dz3[k] - smu : 0.0;
                        rc4[k] = c.f4[j] ? s4[k] * z4[k] + ds4[k] * dz4[k] - smu : 0.0;
                    }
                for (size_t k = 0; k < CX; ++k) {
                    const int r2 = (int)(k % nc);
                    rc5[k] = c.f5[r2] ? s5[k] * z5[k] + ds5[k] * dz5[k] - smu : 0.0;
                    rc6[k] = c.f6[r2] ? s6[k] * z6[k] + ds6[k] * dz6[k] - smu : 0.0;
                }
            }
            /* linear terms after eliminating ds, dz:
             * q = r_x + S1^{-1}(Z1 rp1 - rc1) - S2^{-1}(Z2 rp2 - rc2), likewise r. */
            for (size_t k = 0; k < SX; ++k)
                q[k] = rx[k] + (z1[k] * rp1[k] - rc1[k]) / s1[k] - (z2[k] * rp2[k] - rc2[k]) / s2[k];
            for (int k = 0; k < n; ++k)
                r[k] = ru[k] + (z3[k] * rp3[k] - rc3[k]) / s3[k] - (z4[k] * rp4[k] - rc4[k]) / s4[k];
            if (nc) {   /* general rows: q_t += E' wc_t (t >= 1), r_t += F' wc_t */
                for (size_t k = 0; k < CX; ++k)
                    wc[k] = (z5[k] * rp5[k] - rc5[k]) / s5[k] - (z6[k] * rp6[k] - rc6[k]) / s6[k];
                for (int t = 0; t < N; ++t)
                    cons_tadd(&c, wc + (size_t)t * nc, t >= 1 ? q + (size_t)(t - 1) * ns : NULL, r + t * nu);
            }
            riccati_solve(&c, &f, q, r, rdyn, dx, du, work);
            if (pb->S || nc) {
                /* the LQ subproblem's costate also carries the stage
                 * couplings: S du_t + E' Sigma_c,t (E dx_t + F du_t) */
                memcpy(tmp, q, sizeof(double) * SX);
                for (int t = 0; t < N && nc; ++t) {
                    cons_eval(&c, dx + (size_t)t * ns, du + t * nu, dcv + (size_t)t * nc);
                    for (int r2 = 0; r2 < nc; ++r2) wc[(size_t)t * nc + r2] = sigc[(size_t)t * nc + r2] * dcv[(size_t)t * nc + r2];
                    if (t >= 1) cons_tadd(&c, wc + (size_t)t * nc, tmp + (size_t)(t - 1) * ns, NULL);
                }
                if (pb->S)
                    for (int t = 1; t < N; ++t)
                        for (int a = 0; a < nu; ++a) {
                            const double da = du[t * nu + a];
                            for (int i = 0; i < ns; ++i) tmp[(size_t)(t - 1) * ns + i] += pb->S[i + (size_t)a * ns] * da;
                        }
                adjoint(&c, dx, tmp, sigx, dlam);
            } else {
                adjoint(&c, dx, q, sigx, dlam);
            }
            /* dlam is the costate of the LQ subproblem: it satisfies the
             * linearised state stationarity Qt dx + q + A' dlam_{t+1} - dlam_t = 0. */
            /* ds = -rp - C d(x,u);  dz = -(rc + z ds)/s */
            for (int t = 1; t <= N; ++t)
                for (int i = 0; i < ns; ++i) {
                    size_t k = (size_t)(t - 1) * ns + i;
                    double dxi = dx[(size_t)t * ns + i];
                    if (c.f1[i]) { ds1[k] = -rp1[k] - dxi; dz1[k] = -(rc1[k] + z1[k] * ds1[k]) / s1[k]; }
                    else { ds1[k] = 0; dz1[k] = 0; }
                    if (c.f2[i]) { ds2[k] = -rp2[k] + dxi; dz2[k] = -(rc2[k] + z2[k] * ds2[k]) / s2[k]; }
                    else { ds2[k] = 0; dz2[k] = 0; }
                }
            for (int t = 0; t < N; ++t)
                for (int j = 0; j < nu; ++j) {
                    int k = t * nu + j;
                    if (c.f3[j]) { ds3[k] = -rp3[k] - du[k]; dz3[k] = -(rc3[k] + z3[k] * ds3[k]) / s3[k]; }
                    else { ds3[k] = 0; dz3[k] = 0; }
                    if (c.f4[j]) { ds4[k] = -rp4[k] + du[k]; dz4[k] = -(rc4[k] + z4[k] * ds4[k]) / s4[k]; }
                    else { ds4[k] = 0; dz4[k] = 0; }
                }
            for (int t = 0; t < N && nc; ++t) {
                cons_eval(&c, dx + (size_t)t * ns, du + t * nu, dcv + (size_t)t * nc);
                for (int r2 = 0; r2 < nc; ++r2) {
                    size_t k = (size_t)t * nc + r2;
                    if (c.f5[r2]) { ds5[k] = -rp5[k] - dcv[k]; dz5[k] = -(rc5[k] + z5[k] * ds5[k]) / s5[k]; }
                    else { ds5[k] = 0; dz5[k] = 0; }
                    if (c.f6[r2]) { ds6[k] = -rp6[k] + dcv[k]; dz6[k] = -(rc6[k] + z6[k] * ds6[k]) / s6[k]; }
                    else { ds6[k] = 0; dz6[k] = 0; }
                }
            }
            /* largest step to the boundary of s >= 0, z >= 0 */
            double amax = INFINITY;
#define RATIO(v, dv) do { if ((dv) < 0.0) { double rr = -(v) / (dv); if (rr < amax) amax = rr; } } while (0)
            for (size_t k = 0; k < SX; ++k) {
                RATIO(s1[k], ds1[k]); RATIO(z1[k], dz1[k]);
                RATIO(s2[k], ds2[k]); RATIO(z2[k], dz2[k]);
            }
            for (int k = 0; k < n; ++k) {
                RATIO(s3[k], ds3[k]); RATIO(z3[k], dz3[k]);
                RATIO(s4[k], ds4[k]); RATIO(z4[k], dz4[k]);
            }
            for (size_t k = 0; k < CX; ++k) {
                RATIO(s5[k], ds5[k]); RATIO(z5[k], dz5[k]);
                RATIO(s6[k], ds6[k]); RATIO(z6[k], dz6[k]);
            }
#undef RATIO
            if (pass == 0) {
                alpha_aff = fmin(1.0, amax);
                double szaff = 0.0;
                for (int t = 1; t <= N; ++t)
                    for (int i = 0; i < ns; ++i) {
                        size_t k = (size_t)(t - 1) * ns + i;
                        if (c.f1[i]) szaff += (s1[k] + alpha_aff * ds1[k]) * (z1[k] + alpha_aff * dz1[k]);
                        if (c.f2[i]) szaff += (s2[k] + alpha_aff * ds2[k]) * (z2[k] + alpha_aff * dz2[k]);
                    }
                for (int t = 0; t < N; ++t)
                    for (int j = 0; j < nu; ++j) {
                        int k = t * nu + j;
                        if (c.f3[j]) szaff += (s3[k] + alpha_aff * ds3[k]) * (z3[k] + alpha_aff * dz3[k]);
                        if (c.f4[j]) szaff += (s4[k] + alpha_aff * ds4[k]) * (z4[k] + alpha_aff * dz4[k]);
                    }
                for (size_t k = 0; k < CX; ++k) {
                    const int r2 = (int)(k % nc);
                    if (c.f5[r2]) szaff += (s5[k] + alpha_aff * ds5[k]) * (z5[k] + alpha_aff * dz5[k]);
                    if (c.f6[r2]) szaff += (s6[k] + alpha_aff * ds6[k]) * (z6[k] + alpha_aff * dz6[k]);
                }
                double mu_aff = c.m > 0 ? szaff / c.m : 0.0;
                sigma = mu > 0.0 ? pow(mu_aff / mu, 3.0) : 0.0;
            } else {
                alpha = fmin(1.0, tau * amax);
            }
        }
        if (trace) {
            double* tr = trace + (size_t)it * ORC_TRACE_W;
            tr[3] = alpha_aff; tr[4] = sigma; tr[5] = alpha;
        }
        /* update every variable with the one step length */
        for (int k = 0; k < n; ++k) u[k] += alpha * du[k];
        for (size_t k = ns; k < XT; ++k) x[k] += alpha * dx[k];
        for (size_t k = ns; k < XT; ++k) lam[k] += alpha * dlam[k];
        for (size_t k = 0; k < SX; ++k) {
            s1[k] += alpha * ds1[k]; s2[k] += alpha * ds2[k];
            z1[k] += alpha * dz1[k]; z2[k] += alpha * dz2[k];
        }
        for (int k = 0; k < n; ++k) {
            s3[k] += alpha * ds3[k]; s4[k] += alpha * ds4[k];
            z3[k] += alpha * dz3[k]; z4[k] += alpha * dz4[k];
        }
        for (size_t k = 0; k < CX; ++k) {
            s5[k] += alpha * ds5[k]; s6[k] += alpha * ds6[k];
            z5[k] += alpha * dz5[k]; z6[k] += alpha * dz6[k];
        }
    }

    if (u_out) memcpy(u_out, u, sizeof(double) * n);
    if (x_out) memcpy(x_out, x + ns, sizeof(double) * SX);
    if (z_out) {
        memcpy(z_out, z1, 8 * SX); memcpy(z_out + SX, z2, 8 * SX);
        memcpy(z_out + 2 * SX, z3, 8 * (size_t)n); memcpy(z_out + 2 * SX + n, z4, 8 * (size_t)n);
        if (CX) {
            memcpy(z_out + 2 * SX + 2 * (size_t)n, z5, 8 * CX);
            memcpy(z_out + 2 * SX + 2 * (size_t)n + CX, z6, 8 * CX);
        }
    }
    if (st) {
        st->iters = it; st->status = status; st->mu = mu;
        st->res_d = res_d; st->res_p = res_p; st->res = res;
        st->hnorm = hnorm; st->dnorm = dnorm; st->m = c.m;
    }

    free(c.f1); free(c.f2); free(c.f3); free(c.f4); free(c.f5); free(c.f6);
    free(cv); free(s5); free(z5); free(s6); free(z6); free(rp5); free(rp6); free(rc5); free(rc6);
    free(ds5); free(dz5); free(ds6); free(dz6); free(sigc); free(wc); free(dcv);
    free(u); free(x); free(lam); free(s1); free(s2); free(z1); free(z2);
    free(s3); free(s4); free(z3); free(z4); free(rx); free(ru); free(rdyn);
    free(rp1); free(rp2); free(rp3); free(rp4); free(sigx); free(sigu); free(q); free(r);
    free(dx); free(du); free(dlam); free(ds1); free(ds2); free(ds3); free(ds4);
    free(dz1); free(dz2); free(dz3); free(dz4); free(rc1); free(rc2); free(rc3); free(rc4);
    free(work); free(tmp);
    free(f.bpat); free(f.hchol); free(f.pe); free(f.P); free(f.Pn); free(f.PA); free(f.PB); free(f.Y);
    return status;
}
