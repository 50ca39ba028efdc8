/*
 * Oracle interface (test infrastructure only: the tests, the smoke check and
 * the benchmark's CPU-baseline leg may call it; the product path never does).
 *
 * Plain FP64 CPU implementation of the LQ-MPC problem of the paper's Eq. 1
 * (cross term S, disturbance w, general constraints E, F, box bounds) solved
 * by Mehrotra's predictor-corrector method on the uncondensed problem, each
 * Newton step by a backward Riccati recursion.  Matrices A, Q, Qf are CSR (row pointers, column indices,
 * values); B (ns x nu) and R (nu x nu) are dense column-major.  Bounds may be
 * +-INFINITY (the constraint is then absent).
 */
#ifndef LQMPC_ORACLE_H
#define LQMPC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOT_PD = 3, ORC_ERR_MAXITER = 4, ORC_ERR_NAN = 6 };
enum { ORC_TRACE_W = 6 };  /* per iteration: mu, res_d, res_p, alpha_aff, sigma, alpha */

typedef struct {
    int ns, nu, N;
    const int* a_ptr; const int* a_idx; const double* a_val;
    const double* B;
    const int* q_ptr; const int* q_idx; const double* q_val;
    const int* qf_ptr; const int* qf_idx; const double* qf_val;
    const double* R;
    const double *xl, *xu, *ul, *uu;
    /* General data of Eq. 1, each optional (NULL / nc = 0: absent):
     *   S  (ns x nu, column-major): cross term x_t' S u_t of the stage cost, t = 0..N-1
     *   w  (N x ns, w_t at w + t*ns): x_{t+1} = A x_t + B u_t + w_t
     *   E (nc x ns), F (nc x nu), column-major, gl, gu (nc, +-INFINITY allowed):
     *       gl <= E x_t + F u_t <= gu for t = 0..N-1 (x_0 = xbar) */
    const double* S;
    const double* w;
    int nc;
    const double *E, *F, *gl, *gu;
} orc_problem;

/* u_init (nullable, nu*N): warm start from this input sequence instead of
 * the box midpoints (the learned warm start; the paper starts cold): clipped
 * into the input box with a margin of 1% of each two-sided range (1e-2 from
 * a one-sided bound), every slack s0 = max(slack, 1e-2) and every dual
 * z0 = mu0 / s0 (mu0 <= 0 selects 1e-2). */
typedef struct { double tol; int max_iter; double tau; const double* u_init; double mu0; } orc_options;

typedef struct {
    int iters, status, m;
    double mu, res_d, res_p, res, hnorm, dnorm;
} orc_stats;

/* u_out: nu*N (u_t at t*nu); x_out: ns*N states x_1..x_N (nullable);
 * z_out: duals [z_xu (ns*N), z_xl (ns*N), z_uu (n), z_ul (n), z_gu (nc*N),
 * z_gl (nc*N)] (nullable);
 * trace: (max_iter+1) x ORC_TRACE_W (nullable).  Returns an ORC_* status. */
int orc_ipm_solve(const orc_problem* pb, const double* xbar, const orc_options* op,
                  double* u_out, double* x_out, double* z_out, orc_stats* st, double* trace);

#ifdef __cplusplus
}
#endif
#endif
