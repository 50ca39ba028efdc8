/*
 * lqmpc: condensed-space interior-point solver for box-constrained
 * linear-quadratic MPC on one B300 GPU (sm_103a).
 *
 * The problem (the paper's Eq. 1; lqmpc_setup takes the box-constrained case
 * S = 0, no general constraints, w = 0, lqmpc_setup_general the rest):
 *     min  1/2 sum_{t=1}^{N-1} x_t' Q x_t + 1/2 x_N' Qf x_N + 1/2 sum_{t=0}^{N-1} u_t' R u_t
 *          + sum_{t=0}^{N-1} x_t' S u_t
 *     s.t. x_0 = x0,  x_{t+1} = A x_t + B u_t + w_t          (t = 0..N-1)
 *          gl <= E x_t + F u_t <= gu                       (t = 0..N-1)
 *          xl <= x_t <= xu  (t = 1..N),  ul <= u_t <= uu  (t = 0..N-1).
 * The states are eliminated once (Section II: x = Phi x0 + Gamma u, Gamma the
 * block lower-triangular Toeplitz matrix of the blocks A^k B), giving the
 * dense QP of Eq. 3 in u (n = nu*N variables).  Each interior-point iteration
 * (Section III, Algorithm 1) forms the condensed KKT matrix of Eq. 7,
 *     M = H + Gamma' Sigma_x Gamma + Sigma_u,
 * factors it by Cholesky, solves for the input step and recovers the slack
 * and dual steps by products with Gamma.
 *
 * Conventions for every entry point:
 *  - Matrices are column-major unless stated.  Sparse matrices are CSR with
 *    int32 row pointers (rows+1), int32 column indices and double values.
 *  - Input vectors are u_t stacked (u[t*nu + c]); state vectors x_1..x_N
 *    stacked (x[(t-1)*ns + i]).
 *  - Pointers are host memory unless the name says "device".  The caller owns
 *    every buffer it passes; the context owns all device memory it allocates.
 *  - No function throws across this boundary or aborts the process.  Errors
 *    are reported as an lqmpc_status; on failure, output buffers hold the best
 *    available values (the last iterate for a solve) or are left untouched
 *    for argument errors.
 *  - Bounds may be -INFINITY / +INFINITY; an infinite bound is absent.
 *  - All device work runs on the stream given at setup.  For NULL the context
 *    creates its own blocking stream, which is ordered with the legacy
 *    default stream both ways (so work the caller puts on the legacy stream
 *    is ordered with the solves) and, unlike the legacy stream, can hold the
 *    captured CUDA graphs the solves replay.  Calls on one context are not
 *    thread-safe.
 *  - There is no CPU fallback: if the CUDA device or kernels are unavailable
 *    the calls return LQMPC_ERR_CUDA.
 */
#ifndef LQMPC_H
#define LQMPC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lqmpc_ctx lqmpc_ctx;

typedef enum {
    LQMPC_OK = 0,
    LQMPC_ERR_ARG = 1,          /* invalid argument (sizes, NULL pointers, NaN data) */
    LQMPC_ERR_CUDA = 2,         /* CUDA runtime error or no usable device */
    LQMPC_ERR_NOT_PD = 3,       /* Cholesky of M failed even in FP64 (Eq. 7 requires M > 0) */
    LQMPC_ERR_MAXITER = 4,      /* iteration limit reached before the stop test */
    LQMPC_ERR_INFEASIBLE = 5,   /* x0 outside its bounds or detected infeasibility */
    LQMPC_ERR_NAN = 6,          /* non-finite iterate */
    LQMPC_ERR_STALL = 7,        /* iterative refinement stalled and fallback disabled */
    LQMPC_ERR_TIMEOUT = 8,      /* a bounded device-side wait gave up */
    LQMPC_ERR_UNSUPPORTED = 9   /* option or size not supported by this build */
} lqmpc_status;

/* Arithmetic of the KKT step (the M formation, factorisation and solves). */
enum {
    LQMPC_FP64 = 0,         /* FP64 SYRK, FP64 Cholesky and solves */
    LQMPC_MIXED_BF16 = 1,   /* BF16 tensor-core SYRK (FP32 accumulate), FP32 Cholesky,
                               FP64 iterative refinement, FP64 fallback */
    LQMPC_MIXED_TF32 = 2,   /* as above with TF32 tensor-core SYRK */
    LQMPC_FP32 = 3,         /* FP32-accurate SYRK (split-TF32 tensor-core products; CUDA cores
                               where tensor maps are unavailable), FP32 Cholesky,
                               FP64 refinement */
    LQMPC_FP32X2 = 4        /* two-level FP32 preconditioner: FP64 formation, FP32 Cholesky
                               L1 of M, then FP32 Cholesky L2 of L1^-1 M L1^-T (formed from
                               E = M - L1 L1' in float-float), preconditioner (L1 L2)^-T (L1 L2)^-1,
                               FP64 refinement; the tier between LQMPC_FP32 and LQMPC_FP64 */
};

typedef struct {
    double tol;          /* stop: max(||r_d||/(1+||h||), ||r_p||/(1+||d||), mu) <= tol; 1e-8 */
    int max_iter;        /* iteration limit; 100 */
    int precision;       /* LQMPC_FP64 (default) / LQMPC_MIXED_BF16 / LQMPC_MIXED_TF32 / LQMPC_FP32 /
                            LQMPC_FP32X2 */
    int refine_max;      /* conjugate-gradient steps per KKT solve with an FP32 factor (30);
                            BF16/TF32 factors get min(refine_max, 12) before escalating */
    double refine_tol;   /* refinement stops at ||b - M du||_inf <= refine_tol ||b||_inf (1e-10)
                            or <= 0.01 tol (1 + ||h||_inf), whichever is larger */
    int fallback;        /* 1: when refinement stalls (two steps that do not halve the residual)
                            or runs out of steps, move to a more accurate factor for the rest of
                            the solve: BF16/TF32 -> FP32 -> FP64 */
    double tau;          /* fraction to the boundary; 0.995 */
    int verbose;         /* 1: keep the per-iteration trace of the last solve */
} lqmpc_options;

typedef struct {
    int iters;           /* interior-point iterations taken */
    int refine_steps;    /* total refinement steps (mixed modes) */
    int fallbacks;       /* precision escalations (BF16/TF32 -> FP32 -> FP32X2 -> FP64) */
    int status;          /* lqmpc_status of the solve */
    double mu;           /* final complementarity s'z/m */
    double res_primal;   /* final ||r_p||_inf/(1+||d||_inf) */
    double res_dual;     /* final ||r_d||_inf/(1+||h||_inf) */
    double t_total_ms;   /* device time of the whole solve (CUDA events) */
    double t_kkt_ms;     /* device time of the KKT steps (form M, factor, solve) */
    double t_syrk_tc_ms; /* device time of the tensor-core SYRK launches (CUDA events) */
    double t_syrk_cc_ms; /* device time of the CUDA-core (FP64/FP32) SYRK launches */
    int syrk_tc_launches;
    int syrk_cc_launches;
    double t_syrk_fp64_ms; /* device time of the FP64 formations of M (FP64 solves and fallbacks) */
    int syrk_fp64_launches;
    double t_syrk_tc3_ms;  /* the split-TF32 (FP32-accurate) share of t_syrk_tc_ms */
    int syrk_tc3_launches;
    double t_potrf32_ms;   /* device time of the low-precision (FP32) Cholesky factorisations */
    int potrf32_launches;
} lqmpc_stats;

/* Default options (values in the comments above). */
lqmpc_options lqmpc_default_options(void);

/* Human-readable name of a status code (static string, never NULL). */
const char* lqmpc_status_str(int status);

/*
 * Build a solver context for one plant: uploads the data, runs the one-time
 * state elimination (Section II: the blocks A^k B of Gamma, in FP64 because
 * powers of A may grow) and forms H = Gamma' Qbar Gamma + Rbar (Eq. 3a).
 *  ns, nu, N   : states, inputs, horizon (all >= 1).
 *  a_*         : A (ns x ns) in CSR.
 *  B           : ns x nu dense column-major.
 *  q_*, qf_*   : Q and Qf (ns x ns) in CSR, symmetric positive semidefinite;
 *                qf_* all NULL means Qf = Q.
 *  R           : nu x nu dense column-major, symmetric positive definite.
 *  xl, xu      : ns state bounds; ul, uu: nu input bounds (+-INFINITY allowed).
 *  opts        : NULL for defaults; copied.
 *  stream      : a cudaStream_t, or NULL (see the stream convention above).
 * Returns LQMPC_ERR_ARG for bad sizes/pointers/NaNs or crossed bounds,
 * LQMPC_ERR_CUDA if the device is unusable.  *out is NULL on failure.
 */
lqmpc_status lqmpc_setup(lqmpc_ctx** out, int ns, int nu, int N,
                         const int* a_ptr, const int* a_idx, const double* a_val,
                         const double* B,
                         const int* q_ptr, const int* q_idx, const double* q_val,
                         const int* qf_ptr, const int* qf_idx, const double* qf_val,
                         const double* R,
                         const double* xl, const double* xu, const double* ul, const double* uu,
                         const lqmpc_options* opts, void* stream);

/* General data of Eq. 1 (Section II).  Every pointer is host memory, owned
 * by the caller and read during the call only; NULL (or nc = 0) means absent. */
typedef struct {
    const double* S;    /* ns x nu column-major: cross term x_t' S u_t of the stage cost;
                           [Q S; S' R] must be positive semidefinite (not checked) */
    const double* w;    /* N x ns, w_t at w + t*ns: known disturbance of the dynamics */
    int nc;             /* general constraint rows per stage */
    const double* E;    /* nc x ns column-major */
    const double* F;    /* nc x nu column-major */
    const double *gl, *gu;  /* nc each: gl <= E x_t + F u_t <= gu (+-INFINITY allowed) */
    const double* K;    /* nu x ns column-major: stabilising feedback of the state
                           elimination, u_t = K x_t + v_t (Section II); the solver then runs in v
                           (A + B K in the powers of the elimination) and returns u */
} lqmpc_general;

/*
 * As lqmpc_setup, for the general problem of Eq. 1.  The general rows are
 * lifted into the state: stage t's rows become nc extra states of x_{t+1}
 * (c_{t+1} = E x_t + F u_t, no cost, bounds [gl, gu]), so the condensed KKT
 * matrix of Eq. 7 carries them in its Gamma' Sigma Gamma term; with K the
 * input bounds become nu more lifted rows (u_t = K x_t + v_t) and v is free.
 * Solves return u in every case.  The stage-level entry points
 * (lqmpc_get_gstack, lqmpc_gamma_mv, lqmpc_form_kkt, lqmpc_get_duals, ...)
 * work on the lifted state of dimension ns + nc (+ nu with K), whose extra
 * rows come after the plant's states; solves read x0 as the plant's ns states
 * (the lifted rows start at zero: no column of the lifted A holds them).
 * With K, warm starts
 * (lqmpc_solve_warm, lqmpc_solve_batch_warm) return LQMPC_ERR_UNSUPPORTED.
 * g = NULL is lqmpc_setup.  LQMPC_ERR_ARG as lqmpc_setup, and for non-finite
 * S, w, E, F, K, crossed or NaN row bounds, or nc > 0 with a NULL array.
 */
lqmpc_status lqmpc_setup_general(lqmpc_ctx** out, int ns, int nu, int N,
                                 const int* a_ptr, const int* a_idx, const double* a_val,
                                 const double* B,
                                 const int* q_ptr, const int* q_idx, const double* q_val,
                                 const int* qf_ptr, const int* qf_idx, const double* qf_val,
                                 const double* R,
                                 const double* xl, const double* xu, const double* ul, const double* uu,
                                 const lqmpc_general* g, const lqmpc_options* opts, void* stream);

/* Replace the options of a context (takes effect at the next solve). */
lqmpc_status lqmpc_set_options(lqmpc_ctx* ctx, const lqmpc_options* opts);

/*
 * Solve the QP for initial state x0 (ns, host) and write the optimal input
 * sequence to u_out (nu*N, host).  Host-to-device and device-to-host copies
 * are part of the call.  stats may be NULL.  Returns the solve status
 * (LQMPC_ERR_INFEASIBLE if the problem has no interior iterate that
 * converges, LQMPC_ERR_MAXITER, LQMPC_ERR_NAN, LQMPC_ERR_NOT_PD).
 */
lqmpc_status lqmpc_solve(lqmpc_ctx* ctx, const double* x0, double* u_out, lqmpc_stats* stats);

/* As lqmpc_solve with x0_device (ns doubles) and u_device (nu*N doubles) in
 * device memory of the context's GPU; no host copies except 'stats'. */
lqmpc_status lqmpc_solve_device(lqmpc_ctx* ctx, const double* x0_device, double* u_device,
                                lqmpc_stats* stats);

/*
 * Warm-started solve (the learned warm start; the paper starts cold): as
 * lqmpc_solve, but the iterations start from the guess u_init (nu*N, host)
 * instead of the box midpoint.  u0 = u_init clipped into the input box with a
 * margin of 1% of each two-sided range (1e-2 from a one-sided bound); x0 =
 * the rollout of u0; every slack s0 = max(slack, 1e-2) and every dual
 * z0 = mu0 / s0, a start centred at complementarity mu0 (mu0 <= 0 selects
 * 1e-2).  Any u_init gives the same optimum (the QP is strictly convex); a
 * good one saves iterations.  LQMPC_ERR_ARG for a non-finite u_init.
 */
lqmpc_status lqmpc_solve_warm(lqmpc_ctx* ctx, const double* x0, const double* u_init, double mu0,
                              double* u_out, lqmpc_stats* stats);

/*
 * Solve `count` independent problems (contexts may differ in ns, nu, N and
 * options other than precision, which is taken from ctxs[0]) in lockstep:
 * every kernel launch of an iteration covers all unfinished instances.
 * x0s[i] / u_outs[i] are host pointers for instance i; stats may be NULL or
 * an array of `count`.  All contexts must have been set up with the same
 * stream argument; the batch runs on ctxs[0]'s stream.
 * Returns LQMPC_OK if every instance converged, otherwise the first failing
 * instance's status.
 */
lqmpc_status lqmpc_solve_batch(lqmpc_ctx* const* ctxs, int count, const double* const* x0s,
                               double* const* u_outs, lqmpc_stats* stats);

/*
 * Warm-started batch (the learned warm start over many initial states; the
 * paper starts cold): as lqmpc_solve_batch, with instance i started from the
 * guess u_inits[i] (nu_i*N_i doubles, host) by the rule of lqmpc_solve_warm
 * (clip into the input box with a margin, rollout, slacks floored at 1e-2,
 * duals mu0 / s; mu0 <= 0 selects 1e-2).  LQMPC_ERR_ARG for a NULL u_inits,
 * a NULL entry, a non-finite guess or a NaN mu0.
 */
lqmpc_status lqmpc_solve_batch_warm(lqmpc_ctx* const* ctxs, int count, const double* const* x0s,
                                    const double* const* u_inits, double mu0, double* const* u_outs,
                                    lqmpc_stats* stats);

/*
 * Autotune the launch shapes of batches like this one (same count and
 * largest ns, nu*N and N): the split-K factor of the CUDA-core SYRK, the
 * Cholesky variant (grid-cooperative over all SMs, or one 8-CTA cluster per
 * instance where the matrix fits distributed shared memory) and the FP64
 * formation of M (SYRK, or the backward recursion over the horizon where
 * setup prepared it for a sparse A), each timed on
 * the device with CUDA events on these contexts' data (a representative
 * Sigma from the cold initial point), best of three.  The decision applies
 * to later lqmpc_solve_batch (and, for count = 1, lqmpc_solve) calls with the
 * same signature.  cache_path (nullable): a text file of earlier decisions,
 * one line per signature; a signature found there is not re-measured, a new
 * one is appended.  Contexts as for lqmpc_solve_batch.
 */
lqmpc_status lqmpc_autotune(lqmpc_ctx* const* ctxs, int count, const char* cache_path);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts); differences around a region count its launches. */
unsigned long long lqmpc_kernel_launches(void);

/* Release a context and all device memory it owns.  NULL is a no-op. */
void lqmpc_free(lqmpc_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Stage-level entry points: each runs one step of the hot path on the GPU on
 * host-provided data and copies the result back (host buffers).  They exist
 * for inspection and parity testing of the individual steps.
 * ------------------------------------------------------------------------ */

/* The blocks G_k = A^k B (k = 0..N-1) built at setup (Section II).  G is
 * N*ns*nu doubles: G_k[i, c] at G[(k*nu + c)*ns + i]. */
lqmpc_status lqmpc_get_gstack(lqmpc_ctx* ctx, double* G);

/* H = Gamma' Qbar Gamma + Rbar (n x n, column-major, FP64) built at setup. */
lqmpc_status lqmpc_get_hessian(lqmpc_ctx* ctx, double* H);

/* out = Gamma v (v: n, out: ns*N) and out = Gamma' w (w: ns*N, out: n), using
 * only the G-stack (the implicit Jacobian of the paper's conclusions), in the
 * arithmetic the context's solves use: FP64 when opts.precision is
 * LQMPC_FP64, float-float (two FP32 words per value, about 2^-44 relative per
 * term) in the mixed-precision modes. */
lqmpc_status lqmpc_gamma_mv(lqmpc_ctx* ctx, const double* v, double* out);
lqmpc_status lqmpc_gamma_tmv(lqmpc_ctx* ctx, const double* w, double* out);

/* Form M = H + Gamma' diag(sigx) Gamma + diag(sigu) (Eq. 7) in the given
 * precision (LQMPC_FP64, LQMPC_MIXED_BF16, LQMPC_MIXED_TF32, LQMPC_FP32; or
 * LQMPC_FP32X2: the float-float Horner chains over the horizon that tier
 * uses, available when the context forms FP64 matrices by the chains, else
 * LQMPC_ERR_UNSUPPORTED) and return it as n x n doubles (full symmetric).
 * sigx: ns*N, sigu: n, >= 0. */
lqmpc_status lqmpc_form_kkt(lqmpc_ctx* ctx, const double* sigx, const double* sigu,
                            int precision, double* M);

/* Allocation-free FP64 formation of the same M (the paper has no counterpart:
 * this is a library facility, not a step of the method).
 *
 * For callers that must not allocate device memory while they run: a
 * real-time control loop that cannot take the allocator's latency or the
 * device-wide synchronisation cudaMalloc/cudaFree may imply, or a process
 * whose device memory is entirely held by another allocator.  After the
 * first call on a device (below) a call allocates nothing, host or device:
 * the split-K partial tiles live in one fixed 16 MiB device array inside this
 * library (one per device), and everything else is the context's (G-stack and
 * H from setup) or the caller's.
 *
 * sigx: device pointer, ns*N doubles (stage r, state i at r*ns + i); sigu:
 * device pointer, n doubles; M: device pointer, n*n doubles, receives the
 * full symmetric M column-major.  All three 8-byte aligned and owned by the
 * caller.  Sigma must be finite and >= 0; device data are not inspected.
 * The work is enqueued on the context's stream and the call returns without
 * waiting: synchronise that stream before reading M.
 *
 * The first call on a device sets that device up, with it current: it loads
 * this entry point's two kernels onto the device (under CUDA's default lazy
 * module loading, that is when the CUDA driver places the 16 MiB array in
 * device memory, and it may synchronise the device), looks up the array's
 * address (cudaGetSymbolAddress) and reads the SM count.  Make that first call
 * during set-up, before the loop that must not allocate, and outside any
 * stream capture (with CUDA_MODULE_LOADING=EAGER the array is placed when the
 * CUDA context is created instead).  All calls on a device share the array, so
 * calls whose work overlaps in time (different streams, or different host
 * threads) race and corrupt each other's results: order them.  No part of
 * the array needs to start at zero (every partial is written before it is
 * read), so nothing is cleared between calls.
 *
 * Size limit: n = nu*N <= 1984 (one split of every 64 x 64 lower tile of M
 * must fit in the array); larger contexts get LQMPC_ERR_UNSUPPORTED, with a
 * message on stderr when opts.verbose is set, and nothing is launched.
 * NULL or misaligned pointers give LQMPC_ERR_ARG; a failed launch or
 * address lookup LQMPC_ERR_CUDA. */
lqmpc_status lqmpc_form_kkt_noalloc(lqmpc_ctx* ctx, const double* sigx, const double* sigu, double* M);

/* Form M as above, Cholesky-factor it and solve M x = b (mixed precisions
 * with FP64 iterative refinement).  L (nullable) receives the lower factor
 * as n x n doubles (upper triangle zero); with LQMPC_FP32X2 that is the
 * second-level factor L2 of L1^-1 M L1^-T.  refine_steps (nullable) receives
 * the refinement steps taken.  Returns LQMPC_ERR_NOT_PD if a pivot is not
 * positive, LQMPC_ERR_STALL if refinement did not reach refine_tol. */
lqmpc_status lqmpc_kkt_solve(lqmpc_ctx* ctx, const double* sigx, const double* sigu,
                             int precision, const double* b, double* x, double* L,
                             int* refine_steps);

/* Per-iteration trace of the last solve: rows of 8 doubles (mu, res_dual,
 * res_primal, alpha_aff, sigma, alpha, refinement steps, KKT precision code
 * of the iteration); writes at most max_rows rows and returns the row count
 * in *rows. */
lqmpc_status lqmpc_get_trace(lqmpc_ctx* ctx, double* trace, int max_rows, int* rows);

/* Final duals of the last solve: [z_xu (ns*N), z_xl (ns*N), z_uu (n), z_ul (n)]. */
lqmpc_status lqmpc_get_duals(lqmpc_ctx* ctx, double* z);

/* ---------------------------------------------------------------------------
 * Warm-start network (not in the paper): an MLP
 *     x0 -> GELU(W1 x0 + b1) -> GELU(W2 . + b2) -> W3 . + b3 -> clamp to [lo, hi]
 * mapping an initial state to an input sequence, trained on (x0, u*) pairs
 * with Adam on the mean squared error, its products on the tcgen05 tensor
 * cores in BF16 with FP32 accumulation (FP32 master weights).  GELU is the
 * erf form.  Parameters are exchanged as one FP32 array in the order
 * W1 (n_hidden x n_in, row-major), b1, W2 (n_hidden x n_hidden), b2,
 * W3 (n_out x n_hidden), b3.  All calls run on the network's stream (NULL:
 * an own blocking stream, as for contexts) and return when done.
 * ------------------------------------------------------------------------ */
typedef struct lqmpc_mlp lqmpc_mlp;

/* Create a network; weights and biases ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in))
 * from `seed`.  n_hidden must be a multiple of 128; batches of up to
 * max_batch rows.  Output bounds start at (-inf, inf). */
lqmpc_status lqmpc_mlp_create(lqmpc_mlp** out, int n_in, int n_hidden, int n_out, int max_batch,
                              unsigned long long seed, void* stream);

/* Projection box of the outputs (n_out each, lo <= hi). */
lqmpc_status lqmpc_mlp_set_bounds(lqmpc_mlp* mlp, const double* lo, const double* hi);

/* Copy the FP32 master parameters out / in (set also resets Adam's state). */
lqmpc_status lqmpc_mlp_get_params(lqmpc_mlp* mlp, float* params);
lqmpc_status lqmpc_mlp_set_params(lqmpc_mlp* mlp, const float* params);

/* One forward and backward pass without an update: grads (same layout as
 * the parameters) of L = mean over the B x n_out entries of (y - U)^2 at the
 * unprojected output y; *loss = L.  X: B x n_in, U: B x n_out, FP32 host. */
lqmpc_status lqmpc_mlp_grad(lqmpc_mlp* mlp, const float* X, const float* U, int B, float* grads,
                            double* loss);

/* Train for `epochs` passes over S samples (X: S x n_in, U: S x n_out, FP32
 * host) in shuffled minibatches of `batch` (the last partial batch of an
 * epoch is dropped), Adam (beta1 0.9, beta2 0.999, eps 1e-8) with step size
 * lr.  epoch_loss (nullable, `epochs` entries) receives each epoch's mean
 * training loss.  One training step is captured as a CUDA graph and
 * replayed (LQMPC_GRAPH=0 launches directly). */
lqmpc_status lqmpc_mlp_train(lqmpc_mlp* mlp, const float* X, const float* U, int S, int epochs, int batch,
                             float lr, unsigned long long seed, double* epoch_loss);

/* Projected outputs for `count` inputs (x: count x n_in, u_out: count x
 * n_out, FP64 host); the inputs are rounded to BF16 like the training data. */
lqmpc_status lqmpc_mlp_infer(lqmpc_mlp* mlp, const double* x, int count, double* u_out);

/* Release a network (NULL is a no-op). */
void lqmpc_mlp_free(lqmpc_mlp* mlp);

#ifdef __cplusplus
}
#endif
#endif /* LQMPC_H */
