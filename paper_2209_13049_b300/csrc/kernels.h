// Host-side launchers of the lqmpc kernels (all take a device array of
// instance descriptors; grid.y = instance).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

namespace lqmpc {

struct Inst;

// kernels_ipm.cu
void launch_set_u0(const Inst* d_insts, int count, int max_n, cudaStream_t st);
void launch_init_point(const Inst* d_insts, int count, int max_total, int max_n, double tol,
                       double tau, int max_iter, double refine_tol, cudaStream_t st);
void launch_resid_check(const Inst* d_insts, int count, int max_total, int max_n, int trace_on,
                        cudaStream_t st, bool do_resid, bool do_rd);
void launch_aff(const Inst* d_insts, int count, int max_total, cudaStream_t st);
void launch_corr(const Inst* d_insts, int count, int max_total, cudaStream_t st);
void launch_rhs(const Inst* d_insts, int count, int max_n, cudaStream_t st);
void launch_step_update(const Inst* d_insts, int count, int max_total, int trace_on, int prec,
                        cudaStream_t st);

// kernels_gamma.cu
void launch_gstack(const Inst* d_inst, const Inst& h, cudaStream_t st);
void launch_gamma_mv(const Inst* d_insts, int count, int max_ns, int max_N, int in_role,
                     int out_role, int force, cudaStream_t st);
size_t gamma_tmv_part_doubles(int ns, int n, int N);
void launch_gamma_tmv(const Inst* d_insts, int count, int max_ns, int max_N, int max_n,
                      int w0_role, int w1_role, int o0_role, int o1_role, int scale0, int force,
                      cudaStream_t st);
void launch_gamma_mv_ff(const Inst* d_insts, int count, int max_ns, int max_N, int max_n, int in_role,
                        int out_role, int flags, cudaStream_t st);
void launch_gamma_tmv_ff(const Inst* d_insts, int count, int max_ns, int max_N, int max_n, int w0_role,
                         int w1_role, int o0_role, int o1_role, int scale0, int flags, cudaStream_t st);
void launch_ychain(const Inst* d_insts, int count, cudaStream_t st);
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

// kernels_chol.cu
void launch_potrf(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st,
                  int want_inv = 0);
bool launch_potrf_cluster(const Inst* d_insts, int count, int max_n, int fp64, int flags, cudaStream_t st);
void launch_prec_apply(const Inst* d_insts, int count, int max_n, int in_role, int out_role, int flags,
                       cudaStream_t st);
void launch_chol_solve(const Inst* d_insts, int count, int max_n, int fp64, int in_role,
                       int out_role, int force, cudaStream_t st);

// kernels_refine.cu (preconditioned conjugate gradients on M du = b)
void launch_pcg_begin(const Inst* d_insts, int count, cudaStream_t st);
void launch_pcg_matvec(const Inst* d_insts, int count, int max_n, int mode, cudaStream_t st);
void launch_pcg_pinit(const Inst* d_insts, int count, cudaStream_t st);
void launch_pcg_step_update(const Inst* d_insts, int count, int max_total, cudaStream_t st);
void launch_pcg_beta(const Inst* d_insts, int count, cudaStream_t st);
void launch_vec_copy(const Inst* d_insts, int count, int max_len, int src_role, int dst_role,
                     int len_kind, int force, cudaStream_t st);

// kernels_tc.cu (tcgen05 tensor-core SYRK)
int syrk_tc_tiles(int n);
int syrk_tc_splits(int ns, int nu, int N);
int syrk_tc_plan_partials(int ns, int nu, int N);
std::vector<int> syrk_tc_make_plan(int ns, int nu, int N);
bool syrk_tc_make_maps(const Inst& h, int tf32, void* map_out /* 128-byte CUtensorMap */);
void launch_syrk_tc(const Inst* d_insts, int count, int max_n, int splits, int tf32,
                    const void* d_maps, int force, cudaStream_t st);

// kernels_noalloc.cu (FP64 KKT formation with split-K partials in a fixed
// device array; returns 0, 1 if n exceeds noalloc_max_n(), 2 on a CUDA error)
int noalloc_max_n();
int launch_form_kkt_noalloc(const double* G, int ldg, const double* H, const double* sigx, const double* sigu,
                            double* M, int ns, int nu, int N, cudaStream_t st);

}  // namespace lqmpc
