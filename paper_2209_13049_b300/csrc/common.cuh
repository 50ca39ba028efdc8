// Shared device-side definitions of the lqmpc CUDA path.
//
// Every kernel processes a batch of independent problem instances: blockIdx.y
// selects the instance, blockIdx.x the work item inside it, so a single solve
// is a batch of one and a batched solve uses the same launches (one launch
// per phase covers every instance; finished instances skip their work).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace lqmpc {

// Every kernel launch of the library goes through LQ_LAUNCH so the process-wide
// launch count (lqmpc_kernel_launches) is exact.
void note_launches(int k);
// With LQMPC_CHECK=1 in the environment every launch is followed by a stream
// synchronisation and an error check that names the failing launch (debug
// aid; off by default).
void check_launch(cudaStream_t st, const char* what, const char* file, int line);
// With LQMPC_PROFILE=1 every launch is bracketed by CUDA events and a
// per-kernel table is printed to stderr after each solve (debug aid).
cudaEvent_t prof_start(cudaStream_t st);
void prof_stop(cudaStream_t st, cudaEvent_t e0, const char* what);
#define LQ_LAUNCH(...)                                               \
    do {                                                             \
        cudaEvent_t lq_e0_ = ::lqmpc::prof_start(st);                \
        __VA_ARGS__;                                                 \
        ::lqmpc::note_launches(1);                                   \
        ::lqmpc::prof_stop(st, lq_e0_, #__VA_ARGS__);                \
        ::lqmpc::check_launch(st, #__VA_ARGS__, __FILE__, __LINE__); \
    } while (0)

// Programmatic dependent launch.  The library's kernels go out with
// programmatic stream serialisation, so a kernel's CTAs can be made resident
// while the kernel before it in the stream drains, and every kernel's first
// statement is pdl_wait(): it returns once the previous grid has completed
// and its writes are visible (at once when the launch had no programmatic
// dependency).  The wait is unconditional and comes before any memory
// access, so stream order holds transitively, as with plain launches.
// No kernel signals its dependents early (griddepcontrol.launch_dependents):
// the next kernel is launched as this one's CTAs exit.  Signalling at the
// start made the C2 solve 8% and the 256-instance batch 12% slower, the
// waiting CTAs taking SM resources from the running kernel.
// LQMPC_PDL=0 in the environment launches without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline void lq_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                   Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

constexpr int kMaxParts = 1024;     // max blocks of a reduction launch per instance
constexpr int kParts = 8;           // reduction slots per instance
constexpr int kTraceW = 8;          // mu, res_d, res_p, alpha_aff, sigma, alpha, refine steps, precision

// Per-instance scalars living in device memory.
struct Scal {
    double mu, mu_aff, sigma, alpha, alpha_aff;
    double hnorm, dnorm, res_d, res_p, res;
    double tol, tau, refine_tol;
    double rnorm0, rnorm, rnorm_prev;   // refinement: ||b||, current and previous ||rho||
    double pcg_rz, pcg_alpha;           // conjugate-gradient scalars r'z and the step
    int m;              // number of finite one-sided constraints
    int done;           // 1 once the stop test passed or the solve failed
    int status;         // lqmpc_status of the solve
    int iter;           // iterations taken
    int max_iter;
    int info;           // Cholesky: first non-positive pivot + 1 (0 = ok)
    int refine_ok;      // refinement converged for the current right-hand side
    int refine_steps;   // refinement steps in total
    int refine_cur;     // refinement steps for the current right-hand side
    int stalled;        // refinement stalled (current right-hand side)
    int fallbacks;      // iterations that fell back to FP64
    int use_fp64;       // sticky: remaining iterations in FP64
    int err;            // device-side error flags (bounded wait timeouts etc.)
    int refine_fail;    // refinement stalled or produced a non-finite residual
    int refine_iter;    // refinement steps in the current interior-point iteration
    int prec_used;      // KKT precision of the current iteration (trace)
    int prec_cur;       // KKT precision of this instance (escalates BF16/TF32 -> FP32 -> FP32X2 -> FP64, sticky)
    int kkt_pending;    // the current KKT solve of this instance is not settled yet
    int refine_budget;  // conjugate-gradient steps allowed for the current right-hand side
    int arrive;         // CTAs of the current launch that finished (last_arrival), 0 between launches
    int pcg_loops;      // passes of the device-side conjugate-gradient loop in the latest solve (instance 0)
    int pcg_pass_total[2];  // passes of the loop graphs since the solve began (instance 0; [FP64 preconditioner])
    int spec_fail;      // a KKT solve of this iteration stayed pending while the host was not looking:
                        // the step and update are skipped and the host repeats the iteration
};

// Device descriptor of one instance (all pointers are device memory).
struct Inst {
    int ns, nu, N, n, SX, ldg;
    int q_diag;                       // Q and Qf diagonal
    int pad0;
    // plant
    const int* a_ptr; const int* a_idx; const double* a_val;
    const int* q_ptr; const int* q_idx; const double* q_val;
    const int* qf_ptr; const int* qf_idx; const double* qf_val;
    const double* B;                  // ns x nu
    const double* R;                  // nu x nu
    const double *xl, *xu, *ul, *uu;
    const double* qd;                 // diag(Q) (ns), when q_diag
    const double* qfd;                // diag(Qf) (ns), when q_diag
    // state elimination (G-stack in reversed block order, column-major, ld = ldg):
    // column (N-1-k)*nu + c holds (A^k B)[:, c]
    double* G64;
    float* G32;                       // FP32 rounding of G64 (also the TF32 operand)
    float* G32lo;                     // G64 - G32 in FP32 (float-float products)
    __nv_bfloat16* G16;
    float* Gt;                        // G64 rounded to TF32 (FP32 storage, low 13 bits zero)
    float* Gtlo;                      // G64 - Gt in FP32 (split-TF32 products)
    double* H64;                      // n x n
    float* H32;                       // n x n
    // per solve
    double *xbar, *y, *h;
    double *u, *x;                    // n, SX (x_1..x_N)
    double *s1, *z1, *s2, *z2;        // SX: upper / lower state bound slacks and duals
    double *s3, *z3, *s4, *z4;        // n:  upper / lower input bound slacks and duals
    double *sigx, *sigu;              // SX, n
    double *sgu, *sgl;                // SX + n: z/s of each row's upper and lower family (rows as row_view)
    double *rsu, *rsl;                // SX + n: 1/s of the families, for the iteration
    double *rpu, *rpl;                // SX + n: primal residuals r_p of the families, for the iteration
    double *rcu, *rcl;                // SX + n: the corrector's r_c of the families
    float* sigx32;                    // N x ldg: FP32 Sigma_x, row r at r*ldg, zero padding
    double *wz, *wx;                  // SX: vectors for Gamma' products
    double *wzu, *wxu;                // n
    double *gz, *gw;                  // n: Gamma' outputs
    double *rd, *b, *du;              // n: r_d, right-hand side, the latest KKT solve's du
    double* du_aff;                   // n: a warm start's guess, staged
    double *ds1, *dz1, *ds2, *dz2;    // SX
    double *ds3, *dz3, *ds4, *dz4;    // n
    double* M64; float* M32;          // n x n
    float* Xinv32;                    // n x n: inverse of the FP32 Cholesky factor (preconditioner)
    double* ldiag;                    // 2 x 32 x 32: factored diagonal blocks in flight (cooperative potrf)
    float* ffw;                       // 4 x SX: float-float split of the Gamma' operands (hi0, lo0, hi1, lo1)
    float* ffv;                       // 2 x n: float-float split of the Gamma operand (hi, lo)
    const int* at_ptr; const int* at_idx; const double* at_val;   // A' in CSR (the columns of A)
    const int* bc_ptr; const int* bc_idx; const double* bc_val;   // nonzeros of B per column
    const int* at_pack;               // A' nonzeros packed as (column index, hi bits, lo bits, 0): float-float chains
    const float* bc_ff;               // B's nonzeros split hi + lo (hi plane, then lo plane)
    float* sig_ff;                    // Sigma_x split hi + lo (SX each) for the float-float Horner chains
    float* XinvT32;                   // its transpose (coalesced rows)
    float* Tinv32;                    // n x n scratch of the inversion
    double *rho, *dcorr;              // refinement: residual, correction (n)
    double* mv;                       // n: Gamma' output of matrix-free products
    double *pp, *qq;                  // n: conjugate-gradient direction p and M p
    double* dxs;                      // SX: Gamma du of the latest KKT solve
    double* tmpx;                     // SX scratch
    double* gpart;                    // Gamma' stage-1 partial sums
    float* r32;                       // n FP32 right-hand side
    float *Xlo32, *XloT32;            // two-level tier: low parts of the combined inverse and its transpose (n x n)
    float* r32lo;                     // two-level tier: low part of the preconditioner's intermediate vector (n)
    void* syrk_ws;                    // split-K partial tiles
    size_t syrk_ws_bytes;
    const int* tc_plan;               // tensor-core SYRK: per lower tile (splits, first partial)
    double* part;                     // kParts x kMaxParts reduction partials
    unsigned* bar;                    // grid-barrier state (2 words), queued Cholesky tickets (2 words),
                                      // device-side conjugate-gradient loop count (1 word)
    int* pflags;                      // dataflow Cholesky: epoch, finished tasks, flag per (block column, row block)
    int* mvcnt;                       // float-float Gamma v: arrivals per (r-tile, state tile), 0 between launches
    const int* ftasks;                // queued dataflow Cholesky: task list of this instance alone
    Scal* sc;
    double* trace;                    // (max_iter+1) x kTraceW
    // general data of Eq. 1 (nullptr: absent): cross term S of the stage cost
    // (ns x nu, column-major) and disturbance w (N x ns, w_t at t*ns)
    const double* Sx;
    const double* wd;
};

// Vectors addressed by role, so one launch can name "the same vector" of
// every instance of a batch.
enum Role : int {
    R_U = 0, R_X, R_Y, R_H, R_TMPX, R_WZ, R_WX, R_GZ, R_GW, R_DU, R_RHO, R_DCORR, R_B, R_RD, R_MV, R_P, R_Q, R_DXS, R_NONE
};

__device__ __forceinline__ double* role_ptr(const Inst& I, int r) {
    switch (r) {
        case R_U: return I.u;        case R_X: return I.x;        case R_Y: return I.y;
        case R_H: return I.h;        case R_TMPX: return I.tmpx;  case R_WZ: return I.wz;
        case R_WX: return I.wx;      case R_GZ: return I.gz;      case R_GW: return I.gw;
        case R_DU: return I.du;      case R_RHO: return I.rho;    case R_DCORR: return I.dcorr;
        case R_B: return I.b;        case R_RD: return I.rd;      case R_MV: return I.mv;
        case R_P: return I.pp;       case R_Q: return I.qq;       case R_DXS: return I.dxs;
        default: return nullptr;
    }
}

// Launch predicates: F_FORCE runs even after the instance finished (setup and
// stage-level calls); F_SKIP_REFINED skips instances whose refinement converged
// (or failed); F_PENDING skips instances whose KKT solve is settled; a
// precision mask (bits 8-11, bit p for precision code p) keeps only the
// instances currently at one of those precisions.
// F_N_LE_512 / F_N_GT_512 keep only the instances with n <= 512 / n > 512 (the
// cluster Cholesky's limit: a batch then factors its small instances in
// clusters and only its large ones with the grid-cooperative kernel).
// Blocks per instance of a grid-stride kernel: `nb` fills the GPU for one
// instance; in a batch the instances share it, so each gets a share of about
// 4096 CTAs in all (at least `lo`): the launch stays a few waves and the CTAs
// of instances a launch skips cost little.
inline int per_instance_blocks(int nb, int count, int lo = 4) {
    if (count <= 1) return nb;
    int share = (4096 + count - 1) / count;
    if (share < lo) share = lo;
    return nb < share ? nb : share;
}

constexpr int kPrecTwoLevel = 4;   // Scal::prec_cur of the two-level FP32 tier (LQMPC_FP32X2)

enum Flags : int { F_NONE = 0, F_FORCE = 1, F_SKIP_REFINED = 2, F_PENDING = 4, F_N_LE_512 = 16, F_N_GT_512 = 32 };
__host__ __device__ constexpr int prec_sel(int mask) { return mask << 8; }

__device__ __forceinline__ bool skip_instance(const Inst& I, int flags) {
    if (!(flags & F_FORCE) && I.sc->done) return true;
    if ((flags & F_SKIP_REFINED) && (I.sc->refine_ok || I.sc->refine_fail)) return true;
    if ((flags & F_PENDING) && !I.sc->kkt_pending) return true;
    const int mask = (flags >> 8) & 31;
    if (mask && !((mask >> I.sc->prec_cur) & 1)) return true;
    if ((flags & F_N_LE_512) && I.n > 512) return true;
    if ((flags & F_N_GT_512) && I.n <= 512) return true;
    return false;
}

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction (blockDim.x multiple of 32, <= 1024); result valid in thread 0.
template <int OP>   // 0 sum, 1 max, 2 min
__device__ __forceinline__ double block_reduce(double v, double* smem32) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = OP == 0 ? warp_sum(v) : OP == 1 ? warp_max(v) : warp_min(v);
    __syncthreads();
    if (lane == 0) smem32[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        double t = lane < nw ? smem32[lane]
                             : (OP == 0 ? 0.0 : OP == 1 ? -INFINITY : INFINITY);
        t = OP == 0 ? warp_sum(t) : OP == 1 ? warp_max(t) : warp_min(t);
        v = t;
    }
    return v;
}

// True in the one CTA of an instance that finishes last in this launch; it
// then sees every other CTA's partial (written before its arrival) and
// resets the counter for the next launch.  Every CTA of the instance must
// call it (the launch predicates are uniform per instance).
__device__ __forceinline__ bool last_arrival(Scal* S) {
    __shared__ int last;
    // the CTA barrier orders every thread's writes before thread 0's
    // acquire-release count; the last CTA's acquire then sees every other
    // CTA's writes, and the second barrier passes that on to its threads
    __syncthreads();
    if (threadIdx.x == 0) {
        int old;
        asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], 1;" : "=r"(old) : "l"(&S->arrive) : "memory");
        last = old == (int)gridDim.x - 1;
        if (last) atomicExch(&S->arrive, 0);
    }
    __syncthreads();
    return last;
}

// Reductions shaped for this part's narrow FP64 pipe (two lanes per clock
// per SM), for the per-row and conjugate-gradient kernels.
//
// block_ext: max (MAX) or min of non-negative doubles (and +inf).  Such
// values order like their bit patterns read as signed 64-bit integers, so the
// comparisons run on the integer pipe and the result is exact.  A positive
// NaN orders above +inf (the max keeps it, the min drops it).
constexpr long long kBitsPosInf = 0x7FF0000000000000LL;
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ long long abs_bits(double v) { return __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL; }

// max of two non-negative values by their bit patterns (a NaN is kept)
__device__ __forceinline__ double max_nonneg(double a, double b) {
    return dbits(a) >= dbits(b) ? a : b;
}

template <bool MAX>
__device__ __forceinline__ long long warp_ext_bits(long long b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = MAX ? (t > b ? t : b) : (t < b ? t : b);
    }
    return b;
}

template <bool MAX>
__device__ __forceinline__ double block_ext(long long b, long long* sm32) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    b = warp_ext_bits<MAX>(b);
    __syncthreads();
    if (lane == 0) sm32[w] = b;
    __syncthreads();
    if (w == 0) b = warp_ext_bits<MAX>(lane < nw ? sm32[lane] : (MAX ? 0LL : kBitsPosInf));
    return __longlong_as_double(b);
}

enum RedKind : int { kSum = 0, kMaxNonneg = 1, kMinNonneg = 2 };

// One warp's reduction of n values src[0..n) (kind as RedKind; strided
// over the lanes, then a shuffle tree; every lane gets the result).
template <bool LDCG>
__device__ __forceinline__ double warp_reduce_span(const double* src, int n, int kind) {
    const int lane = threadIdx.x & 31;
    if (kind == kSum) {
        double t = 0.0;
        for (int i = lane; i < n; i += 32) t += LDCG ? __ldcg(src + i) : src[i];
        return warp_sum(t);
    }
    const bool mx = kind == kMaxNonneg;
    long long b = mx ? 0LL : kBitsPosInf;
    for (int i = lane; i < n; i += 32) {
        const long long x = dbits(LDCG ? __ldcg(src + i) : src[i]);
        b = mx ? (x > b ? x : b) : (x < b ? x : b);
    }
    return __longlong_as_double(mx ? warp_ext_bits<true>(b) : warp_ext_bits<false>(b));
}

// This CTA's partials of K quantities at once: the threads' values staged in
// shared memory (stage holds K x blockDim.x doubles), then warp q (and every
// nw-th warp after it) reduces quantity q into partial slot slot[q].  One
// barrier; call once per kernel.
template <int K>
__device__ __forceinline__ void put_parts(const Inst& I, const double (&v)[K], const int (&slot)[K],
                                          const int (&kind)[K], double* stage) {
#pragma unroll
    for (int q = 0; q < K; ++q) stage[q * blockDim.x + threadIdx.x] = v[q];
    __syncthreads();
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        if (q % nw != w) continue;
        const double r = warp_reduce_span<false>(stage + q * blockDim.x, blockDim.x, kind[q]);
        if ((threadIdx.x & 31) == 0) I.part[slot[q] * kMaxParts + blockIdx.x] = r;
    }
}

// The finish of a reduction (the instance's last CTA, after last_arrival):
// warp q (and every nw-th after it) reduces partial slot slot[q] over the
// nb[q] CTAs of the launch, read past L1, into out[q], in a fixed order.
// Ends with a barrier.
template <int K>
__device__ __forceinline__ void reduce_parts(const Inst& I, const int (&slot)[K], const int (&kind)[K],
                                             const int (&nb)[K], double* out) {
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        if (q % nw != w) continue;
        const double r = warp_reduce_span<true>(I.part + (size_t)slot[q] * kMaxParts, nb[q], kind[q]);
        if ((threadIdx.x & 31) == 0) out[q] = r;
    }
    __syncthreads();
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

}  // namespace lqmpc
