// Host-side launchers of the lqmpc kernels (all take a device array of
// instance descriptors; grid.y = instance).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

namespace lqmpc {

struct Inst;

// kernels_ipm.cu
// SMs of the current device (queried once per process; 1 if the query fails)
int device_sm_count();
void launch_set_u0(const Inst* d_insts, int count, int max_n, cudaStream_t st, int warm = 0);
void launch_init_point(const Inst* d_insts, int count, int max_total, int max_n, double tol,
                       double tau, int max_iter, double refine_tol, int prec, cudaStream_t st, double mu0 = 0.0,
                       double smin = 1.0);
// rd_parts (with do_rd): 1 r_d and the right-hand side, 2 the stop test, 3 both;
// split_w: k_resid also splits wz and wx for a float-float Gamma' product
// launched with kFuseInSplit (k_corr likewise wx)
void launch_resid_check(const Inst* d_insts, int count, int max_total, int max_n, int trace_on,
                        cudaStream_t st, bool do_resid, bool do_rd, int rd_parts = 3, bool split_w = false);
void launch_aff(const Inst* d_insts, int count, int max_total, cudaStream_t st);
void launch_corr(const Inst* d_insts, int count, int max_total, cudaStream_t st, bool split_w = false);
void launch_rhs(const Inst* d_insts, int count, int max_n, cudaStream_t st);
void launch_step_update(const Inst* d_insts, int count, int max_total, int trace_on, cudaStream_t st);

// kernels_gamma.cu
void launch_gstack(const Inst* d_inst, const Inst& h, cudaStream_t st);
void launch_gamma_mv(const Inst* d_insts, int count, int max_ns, int max_N, int in_role,
                     int out_role, int force, cudaStream_t st);
size_t gamma_tmv_part_doubles(int ns, int n, int N);
void launch_gamma_tmv(const Inst* d_insts, int count, int max_ns, int max_N, int max_n,
                      int w0_role, int w1_role, int o0_role, int o1_role, int scale0, int force,
                      cudaStream_t st);
// Fusion options of the float-float Gamma products: the input is already
// split (kFuseInSplit: no split kernel), the Gamma v sum also writes the split
// of Sigma_x (Gamma v) for a following Gamma' product (kFuseOutW) and a copy
// into dxs (kFuseOutDxs); the Gamma' product leaves its partials for a fused
// consumer (kFuseNoSum); with kFuseSumHere the Gamma v product sums its own
// split-K partials (no sum launch); with kFuseRhs the sum of a one-vector
// Gamma' w also forms the corrector's right-hand side b = -r_d + Gamma' w +
// w_u (no k_rhs launch).
enum FuseFlags : int {
    kFuseInSplit = 1, kFuseOutW = 2, kFuseOutDxs = 4, kFuseNoSum = 8, kFuseSumHere = 16, kFuseRhs = 32
};
void launch_gamma_mv_ff(const Inst* d_insts, int count, int max_ns, int max_N, int max_n, int in_role,
                        int out_role, int flags, cudaStream_t st, int fuse = 0);
// split count of the float-float Gamma' product (its partials' layout)
int gamma_tmv_ff_splits(int count, int max_ns, int max_N, int max_n, int NV);
void launch_gamma_tmv_ff(const Inst* d_insts, int count, int max_ns, int max_N, int max_n, int w0_role,
                         int w1_role, int o0_role, int o1_role, int scale0, int flags, cudaStream_t st,
                         int fuse = 0);
void launch_ychain(const Inst* d_insts, int count, cudaStream_t st);
void launch_hess_cross(const Inst* d_inst, int n, cudaStream_t st);
void launch_h_cross(const Inst* d_insts, int count, int max_n, cudaStream_t st);
void launch_qbar_y(const Inst* d_insts, int count, int max_sx, cudaStream_t st);
void launch_q_times_g(const Inst* d_inst, const Inst& h, int use_qf, double* out, cudaStream_t st);

// kernels_syrk.cu
int syrk_cc_tiles(int n);
int syrk_cc_splits(int ns, int nu, int N);
void launch_syrk_cc(const Inst* d_insts, int count, int max_n, int splits, int fp64, int mode,
                    const double* gq, const double* gqf, int force, cudaStream_t st);
void launch_syrk_reduce(const Inst* d_insts, int count, int max_n, int splits, int part_kind,
                        int out_fp64, int base_mode, int add_sigu, int force, void* out_override,
                        cudaStream_t st, double shift = 0.0);
void launch_h_to_f32(const Inst* d_inst, int n, cudaStream_t st);

// kernels_lyap.cu (FP64 KKT matrix by the backward recursion, sparse A)
void launch_kkt_lyap(const Inst* d_insts, int count, int max_ns, int max_nu, int max_N, int flags, cudaStream_t st,
                     double shift = 0.0);
double kkt_cost_syrk(int ns, int nu, int N);
double kkt_cost_lyap(int ns, int nu, int N, long long nnzA, long long nnzB);
// the same chains in float-float (the two-level FP32 tier's M; Sigma_x split into sig_ff first)
void launch_kkt_lyap_ff(const Inst* d_insts, int count, int max_ns, int max_nu, int max_N, int max_sx, int flags,
                        cudaStream_t st, double shift);

// kernels_chol.cu
void launch_potrf(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st,
                  int want_inv = 0, int variant = -1, const int* d_tasks = nullptr, int ntasks = 0);
bool launch_potrf_cluster(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st);
bool potrf_cluster_fits(int max_n);
// kernels_flow.cu (dataflow Cholesky with inverse, one instance, FP32)
bool potrf_flow_fits(int count, int max_n);
bool launch_potrf_flow(const Inst* d_insts, int max_n, int flags, cudaStream_t st);
// queued dataflow Cholesky (FP32 with the inverse, any count, n <= 1024):
// the task list holds flowq_task_count(n) entries per instance, written by
// flowq_tasks(instance index, n, out), largest instances first
// two-level FP32 preconditioner (kernels_x2.cu): M32 = fl(M64) with a
// relative diagonal shift; after the first FP32 factor: E, G = X1 E and
// M32 = I + X1 E X1'; after the second: the combined inverse
void launch_x2_round(const Inst* d_insts, int count, int max_n, int flags, cudaStream_t st, double shift);
void launch_x2_refine(const Inst* d_insts, int count, int max_n, int flags, cudaStream_t st);
void launch_x2_combine(const Inst* d_insts, int count, int max_n, int flags, cudaStream_t st);
bool potrf_flowq_fits(int max_n);
int flowq_task_count(int n);
void flowq_tasks(int q, int n, int* out);
bool launch_potrf_flowq(const Inst* d_insts, const int* d_tasks, int ntasks, int max_n, int flags, cudaStream_t st);
// tail: 0 none; 1 / 2 also the conjugate-gradient direction from z = out
// (p = z / p = z + beta p with r'z) in the same launch; 3 the float-float
// split of out (for a Gamma product launched with kFuseInSplit)
void launch_prec_apply(const Inst* d_insts, int count, int max_n, int in_role, int out_role, int flags,
                       cudaStream_t st, int tail = 0);
void launch_chol_solve(const Inst* d_insts, int count, int max_n, int fp64, int in_role,
                       int out_role, int force, cudaStream_t st);

// kernels_refine.cu (preconditioned conjugate gradients on M du = b; `sel`
// is the launch predicate that picks the instances of the solve)
// loop control of the device-side conjugate-gradient loop (while node of a captured graph)
void launch_pcg_more(const Inst* d_insts, int count, int selr, cudaGraphConditionalHandle h, int cap, int reset, int slot,
                     cudaStream_t st);
void launch_pcg_begin(const Inst* d_insts, int count, int sel, int budget_hi, int budget_lo, int budget_mid,
                      cudaStream_t st);
void launch_pcg_matvec(const Inst* d_insts, int count, int max_n, int mode, int sel, cudaStream_t st);
// The same with mv = Gamma'(Sigma_x Gamma v) summed from the float-float
// partials of the preceding Gamma' product (launched with kFuseNoSum).
void launch_pcg_matvec_ff(const Inst* d_insts, int count, int max_n, int splits, int mode, int sel,
                          cudaStream_t st);
void launch_pcg_pinit(const Inst* d_insts, int count, int sel, cudaStream_t st);
void launch_pcg_step_update(const Inst* d_insts, int count, int max_total, int sel, cudaStream_t st);
void launch_pcg_beta(const Inst* d_insts, int count, int sel, cudaStream_t st);
void launch_kkt_begin(const Inst* d_insts, int count, cudaStream_t st);
void launch_kkt_settle(const Inst* d_insts, int count, cudaStream_t st, int mark);
void launch_vec_copy(const Inst* d_insts, int count, int max_len, int src_role, int dst_role,
                     int len_kind, int force, cudaStream_t st);
void launch_vec_add(const Inst* d_insts, int count, int max_n, int src_role, int dst_role, cudaStream_t st);

// kernels_tc.cu (tcgen05 tensor-core SYRK)
int syrk_tc_tiles(int n);
int syrk_tc_splits(int ns, int nu, int N);
int syrk_tc_plan_partials(int ns, int nu, int N);
std::vector<int> syrk_tc_make_plan(int ns, int nu, int N);
// map kinds: 0 BF16 G-stack, 1 TF32-rounded G-stack, 2 its FP32 low part; three maps per instance
bool syrk_tc_make_maps(const Inst& h, int kind, void* map_out /* 128-byte CUtensorMap */);
// mode: 0 BF16, 1 TF32, 2 split TF32 (FP32-accurate)
void launch_syrk_tc(const Inst* d_insts, int count, int max_n, int splits, int mode,
                    const void* d_maps, int force, cudaStream_t st);

// kernels_noalloc.cu (FP64 KKT formation with split-K partials in a fixed
// device array; returns 0, 1 if n exceeds noalloc_max_n(), 2 on a CUDA error)
int noalloc_max_n();
int launch_form_kkt_noalloc(const double* G, int ldg, const double* H, const double* sigx, const double* sigu,
                            double* M, int ns, int nu, int N, cudaStream_t st);

// kernels_mlp.cu (warm-start network: tcgen05 GEMMs with fused epilogues)
// Epilogue operands of one GEMM C[M x N] = A[M x K] B[N x K]^T: row-major
// outputs of M x N (ld N); transposed BF16 copies N x (ld ldt).
struct GemmEpi {
    int M, N, ldt;
    const float* bias;       // N
    float* zf;               // M x N FP32 (z, y or the weight gradient)
    const float* zin;        // M x N FP32 pre-activations (GELU backward)
    __nv_bfloat16* yb;       // M x N BF16
    __nv_bfloat16* ybt;      // N x ldt BF16
    const float* target;     // M x N FP32 (loss)
    int m_real, n_real;      // rows / columns that carry data
    float gscale;            // loss gradient scale 2 / (B n_out)
    double* loss_part;       // per-CTA partial sums of squares
    const double* lo;        // N projection bounds (inference)
    const double* hi;
    double* out64;           // m_real x n_real FP64 (inference)
    int* err;                // bit 0: a bounded wait gave up
};
enum { EPI_WGRAD = 0, EPI_BIAS_GELU = 1, EPI_BIAS_LOSS = 2, EPI_GELU_BWD = 3, EPI_BIAS_PROJ = 4 };
bool mlp_make_map(void* map_out, const void* base, int rows, int cols);
void mlp_gemm(int epi, const void* mapA, const void* mapB, int M, int N, int K, const GemmEpi& ep, cudaStream_t st);
void mlp_gather(const float* Xs, const float* Us, const int* idx, int B, int Bp, int ldt, int nin, int inp, int nout,
                int outp, __nv_bfloat16* X, __nv_bfloat16* XT, float* T, cudaStream_t st);
void mlp_colsum(const __nv_bfloat16* GT, int F, int Bp, int ldt, float* db, cudaStream_t st);
void mlp_adam(float* w, const float* g, float* m, float* v, size_t count, float lr, float b1, float b2, float eps,
              const int* tstep, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wbt, cudaStream_t st);
void mlp_tick(int* tstep, cudaStream_t st);
void mlp_cast(const float* w, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wbt, cudaStream_t st);
void mlp_load_x(const double* x, int count, int nin, int inp, int Bp, __nv_bfloat16* X, cudaStream_t st);
void mlp_sum(const double* part, int n, double* out, cudaStream_t st);

}  // namespace lqmpc
