/*
 * CPU condensed-dense baseline: the condensed-space interior-point method of
 * Section III run on the host cores (the analogue of the paper's "CPU dense"
 * columns in Tables II-V, which solve the condensed problem with dense
 * Cholesky factorisations on the CPU).  A comparison baseline for the
 * benchmark and its tests; not part of the CUDA product path, which never
 * calls it.
 *
 * Problem: Eq. 1 with S = 0, no general constraints, w = 0, K = 0, eliminated
 * into the dense QP of Eq. 3 in u (n = nu*N): x = y + Gamma u with y the
 * free response of x0 and Gamma the block lower-triangular Toeplitz matrix
 * whose block (r, t) is A^(r-t) B (state x_{r+1}, input u_t).  Gamma is kept
 * implicit, as its N blocks G_k = A^k B (the structure the paper's
 * conclusions point at); products with it and the formation of
 *     M = H + Gamma' Sigma_x Gamma + Sigma_u            (Eq. 7)
 * run block by block.  Each iteration: Mehrotra predictor-corrector with one
 * Cholesky factor of M for both right-hand sides (Eq. 7 read with J' r2:
 * M du = -r_d - J' S^-1 (Z r_p - r_c)), slack and dual steps recovered by
 * products with Gamma (Section III), one step length for all variables.
 * The start, the stop test and the step rule are those of the oracle and the
 * GPU solver, so in exact arithmetic all three take the same iterates.
 *
 * Parallelism: OpenMP over block pairs of M, over output blocks of the Gamma
 * products, over the rows of each Cholesky column block and over the
 * elementwise loops.  No external BLAS.
 */
#include "cpu_dense.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    const cpd_problem* p;
    int ns, nu, N, n;
    size_t SX;
    double* G;      /* N blocks, G_k = A^k B, block k at G + k*ns*nu, column-major ns x nu */
    double* H;      /* n x n column-major (full) */
    double* y;      /* free response x_1..x_N of x0 */
    unsigned char *fxu, *fxl, *fuu, *ful;
    int m;
} cpd_ctx;

/* out = A v (CSR) */
static void csr_mv(int rows, const int* ptr, const int* idx, const double* val, const double* v, double* out) {
    for (int r = 0; r < rows; ++r) {
        double acc = 0.0;
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) acc += val[k] * v[idx[k]];
        out[r] = acc;
    }
}

/* out[r] = sum_{t<=r} G_{r-t} v_t  for state rows r = 0..N-1 (x_{r+1}) */
static void gamma_mv(const cpd_ctx* c, const double* v, double* out) {
    const int ns = c->ns, nu = c->nu, N = c->N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < N; ++r) {
        double* o = out + (size_t)r * ns;
        memset(o, 0, sizeof(double) * ns);
        for (int t = 0; t <= r; ++t) {
            const double* Gk = c->G + (size_t)(r - t) * ns * nu;
            for (int a = 0; a < nu; ++a) {
                const double va = v[t * nu + a];
                if (va == 0.0) continue;
                const double* g = Gk + (size_t)a * ns;
                for (int i = 0; i < ns; ++i) o[i] += g[i] * va;
            }
        }
    }
}

/* out_t = sum_{r>=t} G_{r-t}' w_r */
static void gamma_tmv(const cpd_ctx* c, const double* w, double* out) {
    const int ns = c->ns, nu = c->nu, N = c->N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < N; ++t) {
        for (int a = 0; a < nu; ++a) {
            double acc = 0.0;
            for (int r = t; r < N; ++r) {
                const double* g = c->G + (size_t)(r - t) * ns * nu + (size_t)a * ns;
                const double* wr = w + (size_t)r * ns;
                double s = 0.0;
                for (int i = 0; i < ns; ++i) s += g[i] * wr[i];
                acc += s;
            }
            out[t * nu + a] = acc;
        }
    }
}

/* Block (j, k) (j >= k) of sum_r Gamma_r,j' diag(d_r) Gamma_r,k for d over
 * state rows, added into M (both triangles).  Block rows r >= j contribute
 * G_{r-j}' (diag(d_r) G_{r-k}); the scaled block is made once per r. */
static void syrk_blocks(const cpd_ctx* c, const double* d, double* M) {
    const int ns = c->ns, nu = c->nu, N = c->N, n = c->n;
    const int pairs = N * (N + 1) / 2;
#pragma omp parallel
    {
        double* tmp = malloc(sizeof(double) * (size_t)ns * nu);
        double* acc = malloc(sizeof(double) * (size_t)nu * nu);
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < pairs; ++q) {
            int j = (int)((sqrt(8.0 * q + 1.0) - 1.0) / 2.0);
            while (j * (j + 1) / 2 > q) --j;
            while ((j + 1) * (j + 2) / 2 <= q) ++j;
            const int k = q - j * (j + 1) / 2;
            memset(acc, 0, sizeof(double) * (size_t)nu * nu);
            for (int r = j; r < N; ++r) {
                const double* dr = d + (size_t)r * ns;
                const double* Gb = c->G + (size_t)(r - k) * ns * nu;
                const double* Ga = c->G + (size_t)(r - j) * ns * nu;
                for (int b = 0; b < nu; ++b)
                    for (int i = 0; i < ns; ++i) tmp[(size_t)b * ns + i] = dr[i] * Gb[(size_t)b * ns + i];
                for (int a = 0; a < nu; ++a) {
                    const double* ga = Ga + (size_t)a * ns;
                    for (int b = 0; b < nu; ++b) {
                        const double* tb = tmp + (size_t)b * ns;
                        double s = 0.0;
                        for (int i = 0; i < ns; ++i) s += ga[i] * tb[i];
                        acc[a + (size_t)b * nu] += s;
                    }
                }
            }
            for (int b = 0; b < nu; ++b)
                for (int a = 0; a < nu; ++a) {
                    const int row = j * nu + a, col = k * nu + b;
                    M[row + (size_t)col * n] += acc[a + (size_t)b * nu];
                    if (j != k) M[col + (size_t)row * n] += acc[a + (size_t)b * nu];
                }
        }
        free(tmp);
        free(acc);
    }
}

/* Cholesky M = L L' in place (lower, column-major), blocked right-looking:
 * per block column of kNb, the diagonal block is factored by one thread, the
 * panel below it solved row by row in parallel, and the trailing lower
 * triangle updated column by column in parallel (two parallel regions per
 * block column).  Returns 0, or k+1 for a non-positive k-th pivot. */
enum { kNb = 64 };

static int cholesky(int n, double* M) {
    for (int J = 0; J < n; J += kNb) {
        const int jb = n - J < kNb ? n - J : kNb;
        for (int j = J; j < J + jb; ++j) {       /* diagonal block, left-looking within it */
            double* mj = M + (size_t)j * n;
            for (int k = J; k < j; ++k) {
                const double* mk = M + (size_t)k * n;
                const double l = mk[j];
                for (int i = j; i < J + jb; ++i) mj[i] -= mk[i] * l;
            }
            const double d = mj[j];
            if (!(d > 0.0)) return j + 1;
            const double l = sqrt(d);
            mj[j] = l;
            for (int i = j + 1; i < J + jb; ++i) mj[i] /= l;
        }
        const int r0 = J + jb;
        if (r0 >= n) break;
#pragma omp parallel for schedule(static)
        for (int i = r0; i < n; ++i) {           /* panel: L_iJ = A_iJ L_JJ^-T, one row each */
            for (int j = J; j < J + jb; ++j) {
                double v = M[i + (size_t)j * n];
                for (int k = J; k < j; ++k) v -= M[i + (size_t)k * n] * M[j + (size_t)k * n];
                M[i + (size_t)j * n] = v / M[j + (size_t)j * n];
            }
        }
#pragma omp parallel for schedule(dynamic, 8)
        for (int k = r0; k < n; ++k) {           /* trailing lower triangle, one column each */
            double* mk = M + (size_t)k * n;
            for (int j = J; j < J + jb; ++j) {
                const double* mj = M + (size_t)j * n;
                const double l = mj[k];
                for (int i = k; i < n; ++i) mk[i] -= mj[i] * l;
            }
        }
    }
    return 0;
}

static void chol_solve(int n, const double* L, double* b) {
    for (int j = 0; j < n; ++j) {
        const double v = b[j] / L[j + (size_t)j * n];
        b[j] = v;
        for (int i = j + 1; i < n; ++i) b[i] -= L[i + (size_t)j * n] * v;
    }
    for (int j = n - 1; j >= 0; --j) {
        const double* lj = L + (size_t)j * n;
        double v = b[j];
        for (int i = j + 1; i < n; ++i) v -= lj[i] * b[i];
        b[j] = v / lj[j];
    }
}

static double box_mid(double lo, double hi) {
    const int fl = isfinite(lo), fh = isfinite(hi);
    if (fl && fh) return 0.5 * (lo + hi);
    if (fl) return lo + 1.0;
    if (fh) return hi - 1.0;
    return 0.0;
}

static double maxabs(const double* v, size_t n) {
    double m = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const double a = fabs(v[i]);
        if (a > m || a != a) m = a;
    }
    return m;
}

/* One-time build: G_k = A^k B and H = Gamma' Qbar Gamma + Rbar. */
static int setup(cpd_ctx* c) {
    const cpd_problem* p = c->p;
    const int ns = c->ns, nu = c->nu, N = c->N, n = c->n;
    c->G = malloc(sizeof(double) * (size_t)N * ns * nu);
    c->H = calloc((size_t)n * n, sizeof(double));
    if (!c->G || !c->H) return CPD_ERR_ARG;
    memcpy(c->G, p->B, sizeof(double) * (size_t)ns * nu);
    for (int k = 1; k < N; ++k)
        for (int a = 0; a < nu; ++a)
            csr_mv(ns, p->a_ptr, p->a_idx, p->a_val, c->G + (size_t)(k - 1) * ns * nu + (size_t)a * ns,
                   c->G + (size_t)k * ns * nu + (size_t)a * ns);
    /* Q Gamma, Qf for the last state row: block (r, t) = W_r G_{r-t} */
    double* QG = malloc(sizeof(double) * (size_t)N * ns * nu);   /* Q G_k */
    double* QfG = malloc(sizeof(double) * (size_t)N * ns * nu);  /* Qf G_k */
    if (!QG || !QfG) { free(QG); free(QfG); return CPD_ERR_ARG; }
#pragma omp parallel for schedule(static)
    for (int q = 0; q < N * nu; ++q) {
        csr_mv(ns, p->q_ptr, p->q_idx, p->q_val, c->G + (size_t)q * ns, QG + (size_t)q * ns);
        csr_mv(ns, p->qf_ptr, p->qf_idx, p->qf_val, c->G + (size_t)q * ns, QfG + (size_t)q * ns);
    }
    /* H_{jk} = sum_{r >= max(j,k)} G_{r-j}' W_r G_{r-k} + [j == k] R */
    const int pairs = N * (N + 1) / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int q = 0; q < pairs; ++q) {
        int j = (int)((sqrt(8.0 * q + 1.0) - 1.0) / 2.0);
        while (j * (j + 1) / 2 > q) --j;
        while ((j + 1) * (j + 2) / 2 <= q) ++j;
        const int k = q - j * (j + 1) / 2;
        for (int a = 0; a < nu; ++a)
            for (int b = 0; b < nu; ++b) {
                double acc = 0.0;
                for (int r = j; r < N; ++r) {
                    const double* ga = c->G + (size_t)(r - j) * ns * nu + (size_t)a * ns;
                    const double* wg = (r == N - 1 ? QfG : QG) + (size_t)(r - k) * ns * nu + (size_t)b * ns;
                    double s = 0.0;
                    for (int i = 0; i < ns; ++i) s += ga[i] * wg[i];
                    acc += s;
                }
                if (j == k) acc += p->R[a + (size_t)b * nu];
                const int row = j * nu + a, col = k * nu + b;
                c->H[row + (size_t)col * n] = acc;
                c->H[col + (size_t)row * n] = acc;
            }
    }
    free(QG);
    free(QfG);
    return CPD_OK;
}

int cpd_solve(const cpd_problem* p, const double* xbar, const cpd_options* op, double* u_out, cpd_stats* st) {
    if (!p || !xbar || !u_out || p->ns < 1 || p->nu < 1 || p->N < 1) return CPD_ERR_ARG;
#ifdef _OPENMP
    if (op && op->threads > 0) omp_set_num_threads(op->threads);
#endif
    cpd_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = p;
    c.ns = p->ns; c.nu = p->nu; c.N = p->N; c.n = p->nu * p->N;
    c.SX = (size_t)p->N * p->ns;
    const int ns = c.ns, nu = c.nu, N = c.N, n = c.n;
    const size_t SX = c.SX;
    const double tol = op ? op->tol : 1e-8, tau = op ? op->tau : 0.995;
    const int max_iter = op ? op->max_iter : 100;
    int status = setup(&c);
    if (status) { free(c.G); free(c.H); return status; }

    c.fxu = malloc(ns); c.fxl = malloc(ns); c.fuu = malloc(nu); c.ful = malloc(nu);
    c.m = 0;
    for (int i = 0; i < ns; ++i) {
        c.fxu[i] = isfinite(p->xu[i]) != 0; c.fxl[i] = isfinite(p->xl[i]) != 0;
        c.m += N * (c.fxu[i] + c.fxl[i]);
    }
    for (int a = 0; a < nu; ++a) {
        c.fuu[a] = isfinite(p->uu[a]) != 0; c.ful[a] = isfinite(p->ul[a]) != 0;
        c.m += N * (c.fuu[a] + c.ful[a]);
    }

    double* y = malloc(sizeof(double) * SX);
    double* h = malloc(sizeof(double) * n);
    double* u = malloc(sizeof(double) * n);
    double* x = malloc(sizeof(double) * SX);
    double *s1 = malloc(8 * SX), *z1 = malloc(8 * SX), *s2 = malloc(8 * SX), *z2 = malloc(8 * SX);
    double *s3 = malloc(8 * (size_t)n), *z3 = malloc(8 * (size_t)n), *s4 = malloc(8 * (size_t)n),
           *z4 = malloc(8 * (size_t)n);
    double *rp1 = malloc(8 * SX), *rp2 = malloc(8 * SX), *rp3 = malloc(8 * (size_t)n), *rp4 = malloc(8 * (size_t)n);
    double *rc1 = malloc(8 * SX), *rc2 = malloc(8 * SX), *rc3 = malloc(8 * (size_t)n), *rc4 = malloc(8 * (size_t)n);
    double *ds1 = malloc(8 * SX), *dz1 = malloc(8 * SX), *ds2 = malloc(8 * SX), *dz2 = malloc(8 * SX);
    double *ds3 = malloc(8 * (size_t)n), *dz3 = malloc(8 * (size_t)n), *ds4 = malloc(8 * (size_t)n),
           *dz4 = malloc(8 * (size_t)n);
    double *wx = malloc(8 * SX), *gw = malloc(8 * (size_t)n), *rd = malloc(8 * (size_t)n);
    double *sigx = malloc(8 * SX), *rhs = malloc(8 * (size_t)n), *du = malloc(8 * (size_t)n), *gdu = malloc(8 * SX);
    double* M = malloc(sizeof(double) * (size_t)n * n);

    /* y = free response; h = Gamma' Qbar y */
    {
        double* cur = malloc(sizeof(double) * ns);
        memcpy(cur, xbar, sizeof(double) * ns);
        for (int r = 0; r < N; ++r) {
            csr_mv(ns, p->a_ptr, p->a_idx, p->a_val, cur, y + (size_t)r * ns);
            memcpy(cur, y + (size_t)r * ns, sizeof(double) * ns);
        }
        free(cur);
        for (int r = 0; r < N; ++r) {
            if (r == N - 1) csr_mv(ns, p->qf_ptr, p->qf_idx, p->qf_val, y + (size_t)r * ns, wx + (size_t)r * ns);
            else csr_mv(ns, p->q_ptr, p->q_idx, p->q_val, y + (size_t)r * ns, wx + (size_t)r * ns);
        }
        gamma_tmv(&c, wx, h);
    }
    double dnorm = 0.0;
    for (int r = 0; r < N; ++r)
        for (int i = 0; i < ns; ++i) {
            const double yi = y[(size_t)r * ns + i];
            if (c.fxu[i] && fabs(p->xu[i] - yi) > dnorm) dnorm = fabs(p->xu[i] - yi);
            if (c.fxl[i] && fabs(yi - p->xl[i]) > dnorm) dnorm = fabs(yi - p->xl[i]);
        }
    for (int a = 0; a < nu; ++a) {
        if (c.fuu[a] && fabs(p->uu[a]) > dnorm) dnorm = fabs(p->uu[a]);
        if (c.ful[a] && fabs(p->ul[a]) > dnorm) dnorm = fabs(p->ul[a]);
    }
    const double hnorm = maxabs(h, n);

    /* start: box midpoints, rollout, s = max(slack, 1), z = 1 (absent: s = 1, z = 0) */
    for (int t = 0; t < N; ++t)
        for (int a = 0; a < nu; ++a) u[t * nu + a] = box_mid(p->ul[a], p->uu[a]);
    gamma_mv(&c, u, x);
    for (size_t k = 0; k < SX; ++k) x[k] += y[k];
    for (size_t k = 0; k < SX; ++k) {
        const int i = (int)(k % ns);
        s1[k] = c.fxu[i] ? fmax(p->xu[i] - x[k], 1.0) : 1.0; z1[k] = c.fxu[i] ? 1.0 : 0.0;
        s2[k] = c.fxl[i] ? fmax(x[k] - p->xl[i], 1.0) : 1.0; z2[k] = c.fxl[i] ? 1.0 : 0.0;
    }
    for (int k = 0; k < n; ++k) {
        const int a = k % nu;
        s3[k] = c.fuu[a] ? fmax(p->uu[a] - u[k], 1.0) : 1.0; z3[k] = c.fuu[a] ? 1.0 : 0.0;
        s4[k] = c.ful[a] ? fmax(u[k] - p->ul[a], 1.0) : 1.0; z4[k] = c.ful[a] ? 1.0 : 0.0;
    }

    int it = 0;
    double mu = 0.0, res_d = 0.0, res_p = 0.0, res = 0.0, t_form = 0.0, t_factor = 0.0;
    for (it = 0;; ++it) {
        /* residuals: r_d = H u + h + Gamma'(z1 - z2) + z3 - z4, r_p per family */
        gamma_mv(&c, u, x);
        double rpmax = 0.0, sz = 0.0;
#pragma omp parallel for reduction(max : rpmax) reduction(+ : sz) schedule(static)
        for (size_t k = 0; k < SX; ++k) {
            const int i = (int)(k % ns);
            const double xi = x[k] + y[k];
            rp1[k] = c.fxu[i] ? xi + s1[k] - p->xu[i] : 0.0;
            rp2[k] = c.fxl[i] ? -xi + s2[k] + p->xl[i] : 0.0;
            rpmax = fmax(rpmax, fmax(fabs(rp1[k]), fabs(rp2[k])));
            sz += (c.fxu[i] ? s1[k] * z1[k] : 0.0) + (c.fxl[i] ? s2[k] * z2[k] : 0.0);
            wx[k] = z1[k] - z2[k];
        }
        for (int k = 0; k < n; ++k) {
            const int a = k % nu;
            rp3[k] = c.fuu[a] ? u[k] + s3[k] - p->uu[a] : 0.0;
            rp4[k] = c.ful[a] ? -u[k] + s4[k] + p->ul[a] : 0.0;
            rpmax = fmax(rpmax, fmax(fabs(rp3[k]), fabs(rp4[k])));
            sz += (c.fuu[a] ? s3[k] * z3[k] : 0.0) + (c.ful[a] ? s4[k] * z4[k] : 0.0);
        }
        gamma_tmv(&c, wx, gw);
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j) {
            double acc = h[j] + gw[j] + z3[j] - z4[j];
            for (int k = 0; k < n; ++k) acc += c.H[j + (size_t)k * n] * u[k];
            rd[j] = acc;
        }
        mu = c.m > 0 ? sz / c.m : 0.0;
        res_d = maxabs(rd, n) / (1.0 + hnorm);
        res_p = rpmax / (1.0 + dnorm);
        res = fmax(fmax(res_d, res_p), mu);
        if (!(res == res)) { status = CPD_ERR_NAN; break; }
        if (res <= tol) break;
        if (it >= max_iter) { status = CPD_ERR_MAXITER; break; }

        /* M = H + Gamma' Sigma_x Gamma + Sigma_u; Cholesky */
        double t0 = 0.0;
#ifdef _OPENMP
        t0 = omp_get_wtime();
#endif
#pragma omp parallel for schedule(static)
        for (size_t k = 0; k < SX; ++k) sigx[k] = z1[k] / s1[k] + z2[k] / s2[k];
        memcpy(M, c.H, sizeof(double) * (size_t)n * n);
        syrk_blocks(&c, sigx, M);
        for (int k = 0; k < n; ++k) M[k + (size_t)k * n] += z3[k] / s3[k] + z4[k] / s4[k];
        double t1 = 0.0;
#ifdef _OPENMP
        t1 = omp_get_wtime();
        t_form += t1 - t0;
#endif
        if (cholesky(n, M)) { status = CPD_ERR_NOT_PD; break; }
#ifdef _OPENMP
        t_factor += omp_get_wtime() - t1;
#endif

        double alpha_aff = 1.0, sigma = 0.0, alpha = 1.0;
        for (int pass = 0; pass < 2; ++pass) {
            const double smu = sigma * mu;
#pragma omp parallel for schedule(static)
            for (size_t k = 0; k < SX; ++k) {
                const int i = (int)(k % ns);
                if (pass == 0) { rc1[k] = s1[k] * z1[k]; rc2[k] = s2[k] * z2[k]; }
                else {
                    rc1[k] = c.fxu[i] ? s1[k] * z1[k] + ds1[k] * dz1[k] - smu : 0.0;
                    rc2[k] = c.fxl[i] ? s2[k] * z2[k] + ds2[k] * dz2[k] - smu : 0.0;
                }
                wx[k] = (z1[k] * rp1[k] - rc1[k]) / s1[k] - (z2[k] * rp2[k] - rc2[k]) / s2[k];
            }
            for (int k = 0; k < n; ++k) {
                const int a = k % nu;
                if (pass == 0) { rc3[k] = s3[k] * z3[k]; rc4[k] = s4[k] * z4[k]; }
                else {
                    rc3[k] = c.fuu[a] ? s3[k] * z3[k] + ds3[k] * dz3[k] - smu : 0.0;
                    rc4[k] = c.ful[a] ? s4[k] * z4[k] + ds4[k] * dz4[k] - smu : 0.0;
                }
            }
            /* M du = -r_d - Gamma' w_x - w_u */
            gamma_tmv(&c, wx, gw);
            for (int k = 0; k < n; ++k)
                rhs[k] = -rd[k] - gw[k] - ((z3[k] * rp3[k] - rc3[k]) / s3[k] - (z4[k] * rp4[k] - rc4[k]) / s4[k]);
            memcpy(du, rhs, sizeof(double) * n);
            chol_solve(n, M, du);
            gamma_mv(&c, du, gdu);
            double amax = INFINITY;
#pragma omp parallel for reduction(min : amax) schedule(static)
            for (size_t k = 0; k < SX; ++k) {
                const int i = (int)(k % ns);
                if (c.fxu[i]) { ds1[k] = -rp1[k] - gdu[k]; dz1[k] = -(rc1[k] + z1[k] * ds1[k]) / s1[k]; }
                else { ds1[k] = 0.0; dz1[k] = 0.0; }
                if (c.fxl[i]) { ds2[k] = -rp2[k] + gdu[k]; dz2[k] = -(rc2[k] + z2[k] * ds2[k]) / s2[k]; }
                else { ds2[k] = 0.0; dz2[k] = 0.0; }
                if (ds1[k] < 0.0) amax = fmin(amax, -s1[k] / ds1[k]);
                if (dz1[k] < 0.0) amax = fmin(amax, -z1[k] / dz1[k]);
                if (ds2[k] < 0.0) amax = fmin(amax, -s2[k] / ds2[k]);
                if (dz2[k] < 0.0) amax = fmin(amax, -z2[k] / dz2[k]);
            }
            for (int k = 0; k < n; ++k) {
                const int a = k % nu;
                if (c.fuu[a]) { ds3[k] = -rp3[k] - du[k]; dz3[k] = -(rc3[k] + z3[k] * ds3[k]) / s3[k]; }
                else { ds3[k] = 0.0; dz3[k] = 0.0; }
                if (c.ful[a]) { ds4[k] = -rp4[k] + du[k]; dz4[k] = -(rc4[k] + z4[k] * ds4[k]) / s4[k]; }
                else { ds4[k] = 0.0; dz4[k] = 0.0; }
                if (ds3[k] < 0.0) amax = fmin(amax, -s3[k] / ds3[k]);
                if (dz3[k] < 0.0) amax = fmin(amax, -z3[k] / dz3[k]);
                if (ds4[k] < 0.0) amax = fmin(amax, -s4[k] / ds4[k]);
                if (dz4[k] < 0.0) amax = fmin(amax, -z4[k] / dz4[k]);
            }
            if (pass == 0) {
                alpha_aff = fmin(1.0, amax);
                double szaff = 0.0;
#pragma omp parallel for reduction(+ : szaff) schedule(static)
                for (size_t k = 0; k < SX; ++k) {
                    const int i = (int)(k % ns);
                    if (c.fxu[i]) szaff += (s1[k] + alpha_aff * ds1[k]) * (z1[k] + alpha_aff * dz1[k]);
                    if (c.fxl[i]) szaff += (s2[k] + alpha_aff * ds2[k]) * (z2[k] + alpha_aff * dz2[k]);
                }
                for (int k = 0; k < n; ++k) {
                    const int a = k % nu;
                    if (c.fuu[a]) szaff += (s3[k] + alpha_aff * ds3[k]) * (z3[k] + alpha_aff * dz3[k]);
                    if (c.ful[a]) szaff += (s4[k] + alpha_aff * ds4[k]) * (z4[k] + alpha_aff * dz4[k]);
                }
                const double mu_aff = c.m > 0 ? szaff / c.m : 0.0;
                sigma = mu > 0.0 ? pow(mu_aff / mu, 3.0) : 0.0;
            } else {
                alpha = fmin(1.0, tau * amax);
            }
        }
        for (int k = 0; k < n; ++k) {
            u[k] += alpha * du[k];
            s3[k] += alpha * ds3[k]; z3[k] += alpha * dz3[k];
            s4[k] += alpha * ds4[k]; z4[k] += alpha * dz4[k];
        }
#pragma omp parallel for schedule(static)
        for (size_t k = 0; k < SX; ++k) {
            s1[k] += alpha * ds1[k]; z1[k] += alpha * dz1[k];
            s2[k] += alpha * ds2[k]; z2[k] += alpha * dz2[k];
        }
    }

    memcpy(u_out, u, sizeof(double) * n);
    if (st) {
        st->iters = it; st->status = status; st->mu = mu; st->res_d = res_d; st->res_p = res_p; st->res = res;
        st->t_form_s = t_form; st->t_factor_s = t_factor;
#ifdef _OPENMP
        st->threads = omp_get_max_threads();
#else
        st->threads = 1;
#endif
    }
    free(y); free(h); free(u); free(x); free(s1); free(z1); free(s2); free(z2); free(s3); free(z3); free(s4);
    free(z4); free(rp1); free(rp2); free(rp3); free(rp4); free(rc1); free(rc2); free(rc3); free(rc4);
    free(ds1); free(dz1); free(ds2); free(dz2); free(ds3); free(dz3); free(ds4); free(dz4); free(wx); free(gw);
    free(rd); free(sigx); free(rhs); free(du); free(gdu); free(M);
    free(c.fxu); free(c.fxl); free(c.fuu); free(c.ful); free(c.G); free(c.H);
    return status;
}
