/*
 * CPU condensed-dense baseline (comparison baseline, not product code): the
 * condensed-space interior-point method of Section III on the host cores,
 * the analogue of the "CPU dense" columns of the paper's Tables II-V.
 *
 * Problem: Eq. 1 with S = 0, no general constraints, w = 0.  A, Q, Qf are
 * CSR (int32 row pointers and column indices, double values); B (ns x nu)
 * and R (nu x nu) are dense column-major; bounds may be +-INFINITY (absent).
 */
#ifndef LQMPC_CPU_DENSE_H
#define LQMPC_CPU_DENSE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { CPD_OK = 0, CPD_ERR_ARG = 1, CPD_ERR_NOT_PD = 3, CPD_ERR_MAXITER = 4, CPD_ERR_NAN = 6 };

typedef struct {
    int ns, nu, N;
    const int* a_ptr; const int* a_idx; const double* a_val;
    const double* B;
    const int* q_ptr; const int* q_idx; const double* q_val;
    const int* qf_ptr; const int* qf_idx; const double* qf_val;
    const double* R;
    const double *xl, *xu, *ul, *uu;
} cpd_problem;

typedef struct { double tol; int max_iter; double tau; int threads; /* <= 0: OpenMP default */ } cpd_options;

typedef struct {
    int iters, status, threads;
    double mu, res_d, res_p, res;
    double t_form_s, t_factor_s;   /* wall time forming M and factoring it, summed over iterations */
} cpd_stats;

/* Solve for initial state xbar (ns); u_out receives nu*N inputs.  Returns a
 * CPD_* status. */
int cpd_solve(const cpd_problem* p, const double* xbar, const cpd_options* op, double* u_out, cpd_stats* st);

#ifdef __cplusplus
}
#endif
#endif
