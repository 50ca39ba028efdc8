// Tensor-core formation of the condensed KKT matrix (Eq. 7) on sm_103a:
//     M_partial(tile a, tile b, split s) = sum_{chunks of s} Gamma_r[:, a]' diag(D_r) Gamma_r[:, b]
// with D = Sigma_x, BF16 (kind::f16) or TF32 (kind::tf32) operands and FP32
// accumulation in tensor memory.
//
// Operands come straight from the G-stack (the implicit Jacobian): row block
// r of Gamma is the column window starting at (N-1-r)*nu of the reversed
// G-stack, so a TMA box at coordinates (i0, (N-1-r)*nu + 128*a) is the K-major
// tile Gamma_r[i0:i0+K, 128a:128a+128]; columns past n and states past ns are
// zero-filled by TMA, which is exactly Gamma's zero upper block triangle and
// the ragged tails.  Only the right operand is scaled by D (one diagonal on
// one side gives Gamma' D Gamma), done in shared memory by four transform
// warps between the TMA arrival and the MMA issue.
//
// Warp roles (64 + 32 kScaleWarps threads): warp 0 TMA producer, warp 1 TMEM
// allocator and single-thread MMA issuer, warps 2 .. the scale transform,
// warps 2-5 also the epilogue (tcgen05.ld of the 128 x 128 FP32 accumulator,
// coalesced column-major store of the partial tile).  Every mbarrier wait is bounded; a wait that gives up
// marks the CTA aborted, drains its own TMA copies (bounded), frees TMEM and
// reports Scal::err.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

constexpr int kTcTile = 128;
constexpr int kTileBytes = kTcTile * 128;          // one operand tile: 128 rows of 128 bytes of K
// MODE 0 BF16, 1 TF32: A + B tiles per stage, 6 stages.  MODE 2 split TF32
// (the FP32-accurate product from hi + lo operands, three TF32 products):
// A_hi, A_lo, B_hi, B_lo per stage, 3 stages.  Both use 192 KB of shared memory.
template <int MODE> struct TcCfg {
    static constexpr int kTiles = MODE == 2 ? 4 : 2;
    static constexpr int kStageBytes = kTiles * kTileBytes;
    static constexpr int kStages = MODE == 2 ? 3 : 6;
};
constexpr int kStagesMax = 6;
// scale-transform warps (warps 2 .. 2 + kScaleWarps - 1; the first four also
// run the epilogue): each of the B tile's 128 rows is scaled by
// kScaleWarps / 4 threads
constexpr int kScaleWarps = 8;
constexpr int kTcThreads = 64 + 32 * kScaleWarps;
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the CTA abort flag) on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// 1-D bulk copy global -> shared (both 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// K-major operand tile, 128-byte swizzle: rows of 128 bytes, 8-row groups of
// 1024 bytes (stride byte offset), descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1u << 46;                 // descriptor version
    d |= (uint64_t)2u << 61;                 // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulate, A/B format (1 = BF16, 2 = TF32),
// both K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_fmt) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(kTcTile >> 3) << 17) |
           ((uint32_t)(kTcTile >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
    if (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
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

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_syrk_tc(const Inst* __restrict__ insts, const CUtensorMap* maps,
                                                     int splits, int flags) {
    pdl_wait();
    constexpr bool TF32 = MODE != 0;
    constexpr int kStages = TcCfg<MODE>::kStages;
    constexpr int kStageBytes = TcCfg<MODE>::kStageBytes;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[kStagesMax], bar_scaled[kStagesMax], bar_empty[kStagesMax], bar_acc;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ int issued_sh;
    __shared__ __align__(16) float Ds[kStagesMax][64];   // Sigma_x segment of each stage

    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, flags) || I.sc->info) return;
    const int n = I.n, ns = I.ns, nu = I.nu, N = I.N;
    const int nt = (n + kTcTile - 1) / kTcTile;
    const int ntiles = nt * (nt + 1) / 2;
    // balanced split-K plan: tile t owns partials [plan[2t+1], plan[2t+1] + plan[2t])
    int tile = 0;
    while (tile < ntiles && blockIdx.x >= I.tc_plan[2 * tile + 1] + I.tc_plan[2 * tile]) ++tile;
    if (tile >= ntiles) return;
    const int nsplit = I.tc_plan[2 * tile], split = blockIdx.x - I.tc_plan[2 * tile + 1];
    (void)splits;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= tile) ++a;
    const int b = tile - a * (a + 1) / 2;
    constexpr int KC = TF32 ? 32 : 64;               // K elements per 128-byte row
    const int rmin = (a * kTcTile) / nu;
    const int nkc = (ns + KC - 1) / KC;
    const long long nchunks = (long long)(N - rmin) * nkc;
    const int c0 = (int)(nchunks * split / nsplit), c1 = (int)(nchunks * (split + 1) / nsplit);
    const int nq = c1 - c0;

    // 1024-byte aligned stage buffers
    unsigned char* sbase = (unsigned char*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per instance: BF16 (hi), TF32, BF16 lo
    const CUtensorMap* map = maps + 3 * blockIdx.y + (TF32 ? 1 : 0);
    const CUtensorMap* map_lo = maps + 3 * blockIdx.y + 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_scaled[s]), 32 * kScaleWarps);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_acc), 1);
        abort_sh = 0;
        issued_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sh)), "r"(kTcTile) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    volatile int* abort_flag = &abort_sh;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int q = 0; q < nq; ++q) {
                const int s = q % kStages, round = q / kStages;
                if (round > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (round - 1) & 1, abort_flag)) break;
                const int ch = c0 + q;
                const int r = rmin + ch / nkc;
                const int i0 = (ch % nkc) * KC;
                const int off = (N - 1 - r) * nu;
                unsigned char* st = sbase + (size_t)s * kStageBytes;
                const uint32_t fb = smem_u32(&bar_full[s]);
                mbar_expect_tx(fb, kStageBytes + KC * 4);
                // stage layout: A (hi), [A lo], B (hi), [B lo]
                tma_load_2d(smem_u32(st), map, i0, off + a * kTcTile, fb);
                if (MODE == 2) {
                    tma_load_2d(smem_u32(st + kTileBytes), map_lo, i0, off + a * kTcTile, fb);
                    tma_load_2d(smem_u32(st + 2 * kTileBytes), map, i0, off + b * kTcTile, fb);
                    tma_load_2d(smem_u32(st + 3 * kTileBytes), map_lo, i0, off + b * kTcTile, fb);
                } else {
                    tma_load_2d(smem_u32(st + kTileBytes), map, i0, off + b * kTcTile, fb);
                }
                // Sigma_x[r, i0 : i0 + KC] (zero-padded rows of ldg floats, 16-byte aligned)
                bulk_load(smem_u32(&Ds[s][0]), I.sigx32 + (size_t)r * I.ldg + i0, KC * 4, fb);
                ++issued;
            }
            issued_sh = issued;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = make_idesc(TF32 ? 2u : 1u);
            bool ok = true;
            for (int q = 0; q < nq; ++q) {
                const int s = q % kStages, round = q / kStages;
                if (!mbar_wait(smem_u32(&bar_scaled[s]), round & 1, abort_flag)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_u32(sbase + (size_t)s * kStageBytes);
                if (MODE == 2) {
                    // A_hi B_hi + A_hi B_lo + A_lo B_hi in TF32: each operand is hi + lo to about
                    // 2^-22 and the dropped A_lo B_lo is about 2^-22 of the product
                    const uint64_t dah = smem_desc_sw128(sa), dal = smem_desc_sw128(sa + kTileBytes);
                    const uint64_t dbh = smem_desc_sw128(sa + 2 * kTileBytes);
                    const uint64_t dbl = smem_desc_sw128(sa + 3 * kTileBytes);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t o = (uint64_t)(2 * k);
                        mma_issue<true>(tmem, dah + o, dbh + o, idesc, (q > 0 || k > 0) ? 1u : 0u);
                        mma_issue<true>(tmem, dah + o, dbl + o, idesc, 1u);
                        mma_issue<true>(tmem, dal + o, dbh + o, idesc, 1u);
                    }
                } else {
                    const uint32_t sb = sa + kTileBytes;
                    const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
                    for (int k = 0; k < 4; ++k)   // 4 MMAs of 32 bytes of K each
                        mma_issue<TF32>(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc,
                                        (q > 0 || k > 0) ? 1u : 0u);
                }
                mma_commit(smem_u32(&bar_empty[s]));
            }
            if (ok && nq > 0) mma_commit(smem_u32(&bar_acc));
        }
    } else {
        // ---------------- scale transform: B tile row t *= D_r[i0 + K]
        constexpr int kParts = kScaleWarps / 4, kChunks = 8 / kParts;   // 16-byte chunks per thread
        const int t = (threadIdx.x - 64) & 127;   // B-tile row
        const int lc0 = ((threadIdx.x - 64) >> 7) * kChunks;
        for (int q = 0; q < nq; ++q) {
            const int s = q % kStages, round = q / kStages;
            if (!mbar_wait(smem_u32(&bar_full[s]), round & 1, abort_flag)) break;
            const float* D = &Ds[s][0];
            unsigned char* rowp = sbase + (size_t)s * kStageBytes + (MODE == 2 ? 2 : 1) * kTileBytes + (size_t)t * 128;
            if (MODE == 2) {
                // B = D (B_hi + B_lo), re-split into TF32 hi + FP32 lo
                unsigned char* rowl = rowp + kTileBytes;
#pragma unroll
                for (int lc = lc0; lc < lc0 + kChunks; ++lc) {
                    const int p = lc ^ (t & 7);
                    float4* ch = reinterpret_cast<float4*>(rowp + p * 16);
                    float4* cl = reinterpret_cast<float4*>(rowl + p * 16);
                    const float4 vh = *ch, vl = *cl;
                    const float4 d = *reinterpret_cast<const float4*>(D + lc * 4);
                    const float x[4] = {(vh.x + vl.x) * d.x, (vh.y + vl.y) * d.y, (vh.z + vl.z) * d.z,
                                        (vh.w + vl.w) * d.w};
                    float h[4], l[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        unsigned tb;
                        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(tb) : "f"(x[u]));
                        h[u] = __uint_as_float(tb);
                        l[u] = x[u] - h[u];
                    }
                    *ch = make_float4(h[0], h[1], h[2], h[3]);
                    *cl = make_float4(l[0], l[1], l[2], l[3]);
                }
            } else {
#pragma unroll
            for (int lc = lc0; lc < lc0 + kChunks; ++lc) {
                const int p = lc ^ (t & 7);
                uint4* cp = reinterpret_cast<uint4*>(rowp + p * 16);
                uint4 v = *cp;
                if (TF32) {
                    const float4 d = *reinterpret_cast<const float4*>(D + lc * 4);
                    float* f = reinterpret_cast<float*>(&v);
                    f[0] *= d.x; f[1] *= d.y; f[2] *= d.z; f[3] *= d.w;
                } else {
                    const float4 d0 = *reinterpret_cast<const float4*>(D + lc * 8);
                    const float4 d1 = *reinterpret_cast<const float4*>(D + lc * 8 + 4);
                    __nv_bfloat162* h2 = reinterpret_cast<__nv_bfloat162*>(&v);
                    float2 f;
                    f = __bfloat1622float2(h2[0]); h2[0] = __floats2bfloat162_rn(f.x * d0.x, f.y * d0.y);
                    f = __bfloat1622float2(h2[1]); h2[1] = __floats2bfloat162_rn(f.x * d0.z, f.y * d0.w);
                    f = __bfloat1622float2(h2[2]); h2[2] = __floats2bfloat162_rn(f.x * d1.x, f.y * d1.y);
                    f = __bfloat1622float2(h2[3]); h2[3] = __floats2bfloat162_rn(f.x * d1.z, f.y * d1.w);
                }
                *cp = v;
            }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&bar_scaled[s]));
        }
        // ---------------- epilogue: TMEM -> partial tile (column-major), warps 2-5
        if (warp >= 6) goto done;
        {
        float* ws = (float*)I.syrk_ws + (size_t)blockIdx.x * kTcTile * kTcTile;
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        bool have = nq > 0 && mbar_wait(smem_u32(&bar_acc), 0, abort_flag);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int cb = 0; cb < kTcTile; cb += 32) {
            float v[32];
            if (have) {
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.0f;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) ws[(size_t)(cb + j) * kTcTile + row] = v[j];
        }
        }
    }
done:
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_sh) {
        // drain this CTA's own TMA copies before the shared memory is released
        if (threadIdx.x == 0) {
            const int issued = issued_sh;
            for (int q = (issued > kStages ? issued - kStages : 0); q < issued; ++q) {
                const int s = q % kStages, round = q / kStages;
                for (uint32_t it = 0; it < kWaitLimit; ++it)
                    if (mbar_try(smem_u32(&bar_full[s]), round & 1)) break;
            }
            atomicOr(&I.sc->err, 1);
        }
        __syncthreads();
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTile) : "memory");
    }
}

// ---------------------------------------------------------------------------

int syrk_tc_tiles(int n) {
    int nt = (n + kTcTile - 1) / kTcTile;
    return nt * (nt + 1) / 2;
}

int syrk_tc_splits(int ns, int nu, int N) {
    int tiles = syrk_tc_tiles(nu * N);
    long long chunks = (long long)N * ((ns + 63) / 64);
    int s = (device_sm_count() + tiles - 1) / tiles;
    if (s > chunks) s = (int)chunks;
    if (s > 128) s = 128;
    return s < 1 ? 1 : s;
}

// Split-K plan of the tensor-core SYRK: lower tile t of the 128-tiling gets
// max(1, G chunks_t / C) CTAs (C = all chunks, G = number of SMs), so the
// grid is about one wave and every CTA gets about the same number of K chunks.
// Layout: plan[2t] = splits, plan[2t+1] = first partial; plan[2 ntiles] = total.
std::vector<int> syrk_tc_make_plan(int ns, int nu, int N) {
    const int n = nu * N, nt = (n + kTcTile - 1) / kTcTile, ntiles = nt * (nt + 1) / 2;
    const long long nkc = (ns + 63) / 64;
    std::vector<long long> ch(ntiles);
    long long C = 0;
    for (int t = 0; t < ntiles; ++t) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= t) ++a;
        const int rmin = (a * kTcTile) / nu;
        ch[t] = (long long)(N - rmin) * nkc;
        C += ch[t];
    }
    const int G = device_sm_count();
    std::vector<int> plan(2 * (size_t)ntiles + 2, 0);
    int off = 0;
    for (int t = 0; t < ntiles; ++t) {
        long long sp = C > 0 ? (long long)G * ch[t] / C : 1;
        if (sp < 1) sp = 1;
        if (sp > ch[t] && ch[t] > 0) sp = ch[t];
        plan[2 * t] = (int)sp;
        plan[2 * t + 1] = off;
        off += (int)sp;
    }
    plan[2 * (size_t)ntiles] = off;
    return plan;
}

int syrk_tc_plan_partials(int ns, int nu, int N) {
    std::vector<int> p = syrk_tc_make_plan(ns, nu, N);
    return p[p.size() - 2];
}

// kind 0: BF16 G-stack, 1: TF32-rounded G-stack, 2: its FP32 low part.
bool syrk_tc_make_maps(const Inst& h, int kind, void* map_out) {
    const int tf32 = kind != 0;
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
    const size_t esz = tf32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)h.ns, (cuuint64_t)h.n};
    cuuint64_t strides[1] = {(cuuint64_t)h.ldg * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)kTcTile};
    cuuint32_t estr[2] = {1, 1};
    void* base = kind == 1 ? (void*)h.Gt : (kind == 2 ? (void*)h.Gtlo : (void*)h.G16);
    CUresult r = encode((CUtensorMap*)map_out, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void launch_syrk_tc(const Inst* d_insts, int count, int max_n, int splits, int mode, const void* d_maps,
                    int flags, cudaStream_t st) {
    dim3 grid(splits, count);   // splits = total partials of the plan
    const CUtensorMap* maps = (const CUtensorMap*)d_maps;
    if (mode == 1) {
        const size_t smem = (size_t)TcCfg<1>::kStages * TcCfg<1>::kStageBytes + 1024;
        cudaFuncSetAttribute(k_syrk_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(lq_pdl(k_syrk_tc<1>, grid, kTcThreads, smem, st, d_insts, maps, splits, flags));
    } else if (mode == 2) {
        const size_t smem = (size_t)TcCfg<2>::kStages * TcCfg<2>::kStageBytes + 1024;
        cudaFuncSetAttribute(k_syrk_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(lq_pdl(k_syrk_tc<2>, grid, kTcThreads, smem, st, d_insts, maps, splits, flags));
    } else {
        const size_t smem = (size_t)TcCfg<0>::kStages * TcCfg<0>::kStageBytes + 1024;
        cudaFuncSetAttribute(k_syrk_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        LQ_LAUNCH(lq_pdl(k_syrk_tc<0>, grid, kTcThreads, smem, st, d_insts, maps, splits, flags));
    }
}

}  // namespace lqmpc
