// The learned warm start's network: an MLP x0 -> GELU(W1 x + b1) ->
// GELU(W2 . + b2) -> W3 . + b3 -> projection onto the input box, trained by
// Adam on the mean squared error to solver solutions u*.  The paper has no
// network; this is the warm-start upgrade of its interior-point method
// (a better starting point for the iterations of Algorithm 1).
//
// Every product is one tcgen05 GEMM C[M x N] = A[M x K] B[N x K]^T with both
// operands K-major BF16 in global memory, loaded by TMA (128-byte swizzle)
// into a 4-stage shared-memory ring, FP32 accumulation in tensor memory, and
// a fused epilogue:
//   EPI_WGRAD     C                      -> FP32 (weight gradients)
//   EPI_BIAS_GELU z = C + b, y = GELU(z) -> z FP32, y BF16 and y^T BF16
//   EPI_BIAS_LOSS y = C + b, g = 2 (y - u*) / (B n_out) on the real rows and
//                 columns -> y FP32, g BF16 and g^T BF16, sum (y - u*)^2
//   EPI_GELU_BWD  g = C * GELU'(z)       -> g BF16 and g^T BF16
//   EPI_BIAS_PROJ y = clamp(C + b, lo, hi) -> FP64 (inference)
// Transposed copies (y^T, g^T, W^T) exist so that every GEMM of the backward
// pass also reads K-major operands.  GELU is the erf form.
//
// Warp roles (192 threads): warp 0 TMA producer, warp 1 TMEM allocation and
// single-thread MMA issue, warps 2-5 epilogue (one TMEM lane quarter each).
// Waits are bounded; a wait that gives up sets the error word and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

namespace {

constexpr int kGT = 128;                       // output tile edge (M and N)
constexpr int kGK = 64;                        // K elements per stage (128 bytes of BF16)
constexpr int kGStages = 4;
constexpr int kGTileBytes = kGT * 128;         // one operand tile per stage
constexpr int kGStageBytes = 2 * kGTileBytes;
constexpr uint32_t kGWait = 1u << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(c) : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t it = 0; it < kGWait; ++it) {
        if (bar_try(b, parity)) return true;
        if ((it & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void bar_expect(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(b)
        : "memory");
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// BF16 x BF16 -> FP32, both K-major, M = N = 128.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGT >> 3) << 17) |
                                ((uint32_t)(kGT >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(kIdescBf16), "r"(accum));
}

__device__ __forceinline__ void mma_commit_to(uint32_t b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z) {
    // d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

}  // namespace

template <int EPI>
__global__ void __launch_bounds__(192, 1) k_mlp_gemm(const __grid_constant__ CUtensorMap mapA,
                                                     const __grid_constant__ CUtensorMap mapB, int K,
                                                     GemmEpi ep) {
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t full[kGStages], empty[kGStages], accb;
    __shared__ uint32_t tbase;
    __shared__ int abort_sh, issued_sh;
    __shared__ double red[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * kGT, m0 = blockIdx.y * kGT;
    const int nq = K / kGK;
    unsigned char* sb = (unsigned char*)(((uintptr_t)gsm + 1023) & ~(uintptr_t)1023);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            bar_init(su32(&full[s]), 1);
            bar_init(su32(&empty[s]), 1);
        }
        bar_init(su32(&accb), 1);
        abort_sh = 0;
        issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tbase)),
                     "r"(kGT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    volatile int* abort_flag = &abort_sh;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int q = 0; q < nq; ++q) {
                const int s = q % kGStages, round = q / kGStages;
                if (round > 0 && !bar_wait(su32(&empty[s]), (round - 1) & 1, abort_flag)) break;
                unsigned char* st = sb + (size_t)s * kGStageBytes;
                const uint32_t fb = su32(&full[s]);
                bar_expect(fb, kGStageBytes);
                tma2d(su32(st), &mapA, q * kGK, m0, fb);
                tma2d(su32(st + kGTileBytes), &mapB, q * kGK, n0, fb);
                ++issued;
            }
            issued_sh = issued;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int q = 0; q < nq; ++q) {
                const int s = q % kGStages, round = q / kGStages;
                if (!bar_wait(su32(&full[s]), round & 1, abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = su32(sb + (size_t)s * kGStageBytes);
                const uint64_t da = desc_sw128(sa), db = desc_sw128(sa + kGTileBytes);
#pragma unroll
                for (int k = 0; k < 4; ++k)      // 4 MMAs of K = 16 (32 bytes) each
                    mma_bf16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), (q > 0 || k > 0) ? 1u : 0u);
                mma_commit_to(su32(&empty[s]));
            }
            if (ok && nq > 0) mma_commit_to(su32(&accb));
        }
    } else {
        const int quarter = warp & 3;
        const int row = m0 + quarter * 32 + lane;
        const bool have = nq > 0 && bar_wait(su32(&accb), 0, abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        double sq = 0.0;
#pragma unroll 1
        for (int cb = 0; cb < kGT; cb += 32) {
            float v[32];
            if (have) {
                tmem_ld_32cols(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.0f;
            }
            const int c0 = n0 + cb;
            const size_t ro = (size_t)row * ep.N + c0;
            if (EPI == EPI_WGRAD) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    *reinterpret_cast<float4*>(ep.zf + ro + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else if (EPI == EPI_BIAS_GELU || EPI == EPI_BIAS_LOSS || EPI == EPI_GELU_BWD) {
                float o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = c0 + j;
                    if (EPI == EPI_BIAS_GELU) {
                        const float z = v[j] + ep.bias[col];
                        v[j] = z;
                        o[j] = gelu(z);
                    } else if (EPI == EPI_BIAS_LOSS) {
                        const float y = v[j] + ep.bias[col];
                        v[j] = y;
                        float g = 0.0f;
                        if (row < ep.m_real && col < ep.n_real) {
                            const float d = y - ep.target[ro + j];
                            sq += (double)d * d;
                            g = ep.gscale * d;
                        }
                        o[j] = g;
                    } else {
                        o[j] = v[j] * gelu_grad(ep.zin[ro + j]);
                    }
                }
                if (EPI != EPI_GELU_BWD) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        *reinterpret_cast<float4*>(ep.zf + ro + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
#pragma unroll
                for (int j = 0; j < 32; j += 8) {
                    __nv_bfloat162 h[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) h[t] = __floats2bfloat162_rn(o[j + 2 * t], o[j + 2 * t + 1]);
                    *reinterpret_cast<uint4*>(ep.yb + ro + j) = *reinterpret_cast<uint4*>(h);
                }
                // transposed copy: for a fixed column the 32 lanes write 32 consecutive rows
#pragma unroll
                for (int j = 0; j < 32; ++j) ep.ybt[(size_t)(c0 + j) * ep.ldt + row] = __float2bfloat16_rn(o[j]);
            } else {   // EPI_BIAS_PROJ
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = c0 + j;
                    if (row < ep.m_real && col < ep.n_real) {
                        double y = (double)(v[j] + ep.bias[col]);
                        y = y < ep.lo[col] ? ep.lo[col] : (y > ep.hi[col] ? ep.hi[col] : y);
                        ep.out64[(size_t)row * ep.n_real + col] = y;
                    }
                }
            }
        }
        if (EPI == EPI_BIAS_LOSS) {
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) red[quarter] = sq;
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (EPI == EPI_BIAS_LOSS && threadIdx.x == 0)
        ep.loss_part[blockIdx.y * gridDim.x + blockIdx.x] = red[0] + red[1] + red[2] + red[3];
    if (abort_sh) {
        if (threadIdx.x == 0) {
            const int issued = issued_sh;
            for (int q = (issued > kGStages ? issued - kGStages : 0); q < issued; ++q) {
                const int s = q % kGStages, round = q / kGStages;
                for (uint32_t it = 0; it < kGWait; ++it)
                    if (bar_try(su32(&full[s]), round & 1)) break;
            }
            atomicOr(ep.err, 1);
        }
        __syncthreads();
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGT) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Elementwise and reduction kernels of a training step.

// Minibatch gather: rows idx[0..B) of the dataset (FP32, S x nin and S x nout)
// into X (BF16, gridDim.y x inp, zero padding) and X^T (inp x ldt), targets
// into T (FP32, gridDim.y x outp).
__global__ void k_mlp_gather(const float* __restrict__ Xs, const float* __restrict__ Us, const int* __restrict__ idx,
                             int B, int ldt, int nin, int inp, int nout, int outp, __nv_bfloat16* __restrict__ X,
                             __nv_bfloat16* __restrict__ XT, float* __restrict__ T) {
    pdl_wait();
    const int r = blockIdx.y;
    const bool real = r < B;
    const size_t src = real ? (size_t)idx[r] : 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < inp; c += gridDim.x * blockDim.x) {
        const float v = (real && c < nin) ? Xs[src * nin + c] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        X[(size_t)r * inp + c] = h;
        XT[(size_t)c * ldt + r] = h;
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < outp; c += gridDim.x * blockDim.x)
        T[(size_t)r * outp + c] = (real && c < nout) ? Us[src * nout + c] : 0.0f;
}

// Bias gradient: db[f] = sum over the batch of G^T[f, :] (one warp per feature).
__global__ void k_mlp_colsum(const __nv_bfloat16* __restrict__ GT, int F, int Bp, int ldt, float* __restrict__ db) {
    pdl_wait();
    const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= F) return;
    float s = 0.0f;
    for (int b = lane; b < Bp; b += 32) s += __bfloat162float(GT[(size_t)f * ldt + b]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[f] = s;
}

// Adam on the FP32 master copy (bias-corrected moments), then the BF16
// working copies W (rows x cols) and W^T (cols x rows) of weight matrices.
__global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, size_t count, float lr, float b1, float b2, float eps,
                           const int* __restrict__ tstep, int rows, int cols, __nv_bfloat16* __restrict__ wb,
                           __nv_bfloat16* __restrict__ wbt) {
    pdl_wait();
    const float t = (float)*tstep;   // steps taken including this one
    const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) {
            const int r = (int)(i / cols), c = (int)(i % cols);
            const __nv_bfloat16 h = __float2bfloat16_rn(wi);
            wb[i] = h;
            wbt[(size_t)c * rows + r] = h;
        }
    }
}

// BF16 working copies of one weight matrix from its FP32 master.
__global__ void k_mlp_cast(const float* __restrict__ w, int rows, int cols, __nv_bfloat16* __restrict__ wb,
                           __nv_bfloat16* __restrict__ wbt) {
    pdl_wait();
    const size_t count = (size_t)rows * cols;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
        wb[i] = h;
        wbt[(size_t)c * rows + r] = h;
    }
}

// FP64 inputs (count x nin) to the BF16 input tile (Bp x inp, zero padding).
__global__ void k_mlp_load_x(const double* __restrict__ x, int count, int nin, int inp, __nv_bfloat16* __restrict__ X) {
    pdl_wait();
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < inp; c += gridDim.x * blockDim.x)
        X[(size_t)r * inp + c] = __float2bfloat16_rn((r < count && c < nin) ? (float)x[(size_t)r * nin + c] : 0.0f);
}

// out += sum of the per-CTA partials (fixed order).
__global__ void k_mlp_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
    pdl_wait();
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_reduce<0>(s, red);
    if (threadIdx.x == 0) *out += s;
}

// ---------------------------------------------------------------------------
// Host side

bool mlp_make_map(void* map_out, const void* base, int rows, int cols) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    // K-major BF16 matrix rows x cols (cols = K, contiguous); box 64 x 128
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGK, (cuuint32_t)kGT};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode((CUtensorMap*)map_out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int EPI>
static void gemm_launch(const void* mapA, const void* mapB, int M, int N, int K, const GemmEpi& ep,
                        cudaStream_t st) {
    const size_t smem = (size_t)kGStages * kGStageBytes + 1024;
    cudaFuncSetAttribute(k_mlp_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const CUtensorMap& a = *reinterpret_cast<const CUtensorMap*>(mapA);
    const CUtensorMap& b = *reinterpret_cast<const CUtensorMap*>(mapB);
    LQ_LAUNCH(lq_pdl(k_mlp_gemm<EPI>, dim3(N / kGT, M / kGT), 192, smem, st, a, b, K, ep));
}

void mlp_gemm(int epi, const void* mapA, const void* mapB, int M, int N, int K, const GemmEpi& ep, cudaStream_t st) {
    switch (epi) {
        case EPI_WGRAD: gemm_launch<EPI_WGRAD>(mapA, mapB, M, N, K, ep, st); break;
        case EPI_BIAS_GELU: gemm_launch<EPI_BIAS_GELU>(mapA, mapB, M, N, K, ep, st); break;
        case EPI_BIAS_LOSS: gemm_launch<EPI_BIAS_LOSS>(mapA, mapB, M, N, K, ep, st); break;
        case EPI_GELU_BWD: gemm_launch<EPI_GELU_BWD>(mapA, mapB, M, N, K, ep, st); break;
        default: gemm_launch<EPI_BIAS_PROJ>(mapA, mapB, M, N, K, ep, st); break;
    }
}

void mlp_gather(const float* Xs, const float* Us, const int* idx, int B, int Bp, int ldt, int nin, int inp, int nout,
                int outp, __nv_bfloat16* X, __nv_bfloat16* XT, float* T, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_mlp_gather, dim3(4, Bp), 256, 0, st, Xs, Us, idx, B, ldt, nin, inp, nout, outp, X, XT, T));
}

void mlp_colsum(const __nv_bfloat16* GT, int F, int Bp, int ldt, float* db, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_mlp_colsum, (F + 7) / 8, 256, 0, st, GT, F, Bp, ldt, db));
}

void mlp_adam(float* w, const float* g, float* m, float* v, size_t count, float lr, float b1, float b2, float eps,
              const int* tstep, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wbt, cudaStream_t st) {
    int nb = (int)((count + 255) / 256);
    nb = nb > 2048 ? 2048 : nb;
    LQ_LAUNCH(lq_pdl(k_mlp_adam, nb, 256, 0, st, w, g, m, v, count, lr, b1, b2, eps, tstep, rows, cols, wb, wbt));
}

__global__ void k_mlp_tick(int* tstep) {
    pdl_wait(); *tstep += 1; }

void mlp_tick(int* tstep, cudaStream_t st) { LQ_LAUNCH(lq_pdl(k_mlp_tick, 1, 1, 0, st, tstep)); }

void mlp_cast(const float* w, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wbt, cudaStream_t st) {
    int nb = (int)(((size_t)rows * cols + 255) / 256);
    nb = nb > 2048 ? 2048 : nb;
    LQ_LAUNCH(lq_pdl(k_mlp_cast, nb, 256, 0, st, w, rows, cols, wb, wbt));
}

void mlp_load_x(const double* x, int count, int nin, int inp, int Bp, __nv_bfloat16* X, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_mlp_load_x, dim3(4, Bp), 256, 0, st, x, count, nin, inp, X));
}

void mlp_sum(const double* part, int n, double* out, cudaStream_t st) {
    LQ_LAUNCH(lq_pdl(k_mlp_sum, 1, 256, 0, st, part, n, out));
}

}  // namespace lqmpc
