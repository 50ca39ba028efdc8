// Condensed KKT matrix on CUDA cores (FP64 and FP32):
//     M = base + Gamma' D Gamma + diag(sigu)           (Eq. 7)
// with D = Sigma_x (the two state-bound families summed) during the
// iterations, or D = diag(Qbar) to form H at setup (Eq. 3a).  A second mode
// takes the right operand from another G-stack-shaped matrix (Q G, Qf G) for a
// non-diagonal Q.
//
// Only the lower triangle of 64 x 64 output tiles is computed.  For a tile
// whose rows are inputs of blocks >= t0, only row blocks r >= t0 of Gamma
// contribute (block lower-triangular structure), so its K range starts there.
// The K range is split across CTAs (split-K); partial tiles go to a
// workspace and a reduce kernel sums them in split order (deterministic),
// adds the base matrix and the diagonal, and writes the full symmetric M.
#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

constexpr int kTile = 64;
constexpr int kKc = 32;

__host__ __device__ inline void tile_of(int t, int& a, int& b) {
    // lower tiles enumerated row by row: t = a(a+1)/2 + b, b <= a
    a = 0;
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    b = t - a * (a + 1) / 2;
}

// mode 0: right operand = D (sigx or its FP32 copy) * G; mode 1: D = qd / qfd
// (setup, H); mode 2: right operand = Q G (r < N-1) or Qf G (r = N-1).
// `force` holds the launch predicate flags (F_FORCE for setup).
template <typename T>
__global__ void __launch_bounds__(256) k_syrk_cc(const Inst* __restrict__ insts, int mode,
                                                 const double* gq, const double* gqf, int splits,
                                                 int force) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, force)) return;
    if (!(force & F_FORCE) && mode == 0 && I.sc->info) return;
    const int n = I.n, ns = I.ns, nu = I.nu, N = I.N, ldg = I.ldg;
    const int nt = (n + kTile - 1) / kTile;
    const int ntiles = nt * (nt + 1) / 2;
    const int tile = blockIdx.x / splits, split = blockIdx.x % splits;
    if (tile >= ntiles) return;
    int a, b;
    tile_of(tile, a, b);
    const int rmin = (a * kTile) / nu;
    const int nkc = (ns + kKc - 1) / kKc;
    const long long nchunks = (long long)(N - rmin) * nkc;
    const long long c0 = nchunks * split / splits, c1 = nchunks * (split + 1) / splits;

    const T* G = sizeof(T) == 8 ? (const T*)I.G64 : (const T*)I.G32;
    __shared__ T As[kKc][kTile + 1];
    __shared__ T Bs[kKc][kTile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0;

    const int lk = threadIdx.x & 31;       // K row this thread loads
    const int lc = threadIdx.x >> 5;       // first column this thread loads (+8 steps)
    for (long long ch = c0; ch < c1; ++ch) {
        const int r = rmin + (int)(ch / nkc);
        const int i0 = (int)(ch % nkc) * kKc;
        const int off = (N - 1 - r) * nu;
        const int i = i0 + lk;
        T d = 0;
        if (i < ns) {
            if (mode == 0) d = sizeof(T) == 8 ? (T)I.sigx[(size_t)r * ns + i] : (T)I.sigx32[(size_t)r * I.ldg + i];
            else if (mode == 1) d = (T)(r == N - 1 ? I.qfd[i] : I.qd[i]);
            else d = 1;
        }
        const double* G2 = (mode == 2) ? (r == N - 1 ? gqf : gq) : nullptr;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = lc + 8 * q;
            const int ca = off + a * kTile + c, cb = off + b * kTile + c;
            T va = 0, vb = 0;
            if (i < ldg) {
                if (ca < n) va = G[(size_t)ldg * ca + i];
                if (cb < n) vb = (mode == 2) ? (T)G2[(size_t)ldg * cb + i] : G[(size_t)ldg * cb + i] * d;
            }
            As[lk][c] = va;
            Bs[lk][c] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKc; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) av[p] = As[kk][ty * 4 + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx * 4 + q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
        }
        __syncthreads();
    }
    T* ws = (T*)I.syrk_ws + ((size_t)tile * splits + split) * kTile * kTile;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) ws[(ty * 4 + p) * kTile + tx * 4 + q] = acc[p][q];
}

// M[j,k] = base[j,k] + sum_s partial_s[max, min] + [j==k] sigu[j].
// base_mode 0: H (FP64 or FP32 copy), 1: Rbar (block diagonal from R), 2: none.
// Tout = double writes M64, float writes M32.  TP is the partial type,
// TILE the tile edge of the partial layout.  LOWER: the lower triangle only
// (the FP32 factorisations read nothing else), with FP32 partials summed in
// float-float (TwoSum) rather than by a dependent chain of FP64 adds.
template <typename TP, typename Tout, int TILE, bool COLMAJOR = false, bool LOWER = false>
__global__ void k_syrk_reduce(const Inst* __restrict__ insts, int splits, int base_mode,
                              int add_sigu, int force, Tout* out_override, double shift) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    if (skip_instance(I, force)) return;
    if (!(force & F_FORCE) && I.sc->info) return;
    const int n = I.n;
    const size_t total = (size_t)n * n;
    Tout* M = out_override ? out_override : (sizeof(Tout) == 8 ? (Tout*)I.M64 : (Tout*)I.M32);
    const TP* ws = (const TP*)I.syrk_ws;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(q % n), k = (int)(q / n);
        if (LOWER && j < k) continue;
        int p = j > k ? j : k, m = j > k ? k : j;
        int a = p / TILE, b = m / TILE;
        int t = a * (a + 1) / 2 + b;
        int first = t * splits, cnt = splits;
        if (COLMAJOR) { cnt = I.tc_plan[2 * t]; first = I.tc_plan[2 * t + 1]; }   // tensor-core plan
        const TP* src = ws + (size_t)first * TILE * TILE +
                        (COLMAJOR ? (m % TILE) * TILE + (p % TILE) : (p % TILE) * TILE + (m % TILE));
        double acc = 0.0;
        if (LOWER && sizeof(TP) == 4) {
            float sh = 0.f, sl = 0.f;
            for (int s = 0; s < cnt; ++s) {
                const float x = (float)src[(size_t)s * TILE * TILE];
                const float t = sh + x;
                const float z = t - sh;
                sl += (sh - (t - z)) + (x - z);
                sh = t;
            }
            acc = (double)sh + (double)sl;
        } else {
            for (int s = 0; s < cnt; ++s) acc += (double)src[(size_t)s * TILE * TILE];
        }
        double base = 0.0;
        if (base_mode == 0) base = sizeof(Tout) == 8 ? I.H64[q] : (double)I.H32[q];
        else if (base_mode == 1) {
            if (j / I.nu == k / I.nu) base = I.R[(j % I.nu) + I.nu * (k % I.nu)];
        }
        double v = base + acc;
        if (add_sigu && j == k) v += I.sigu[j];
        if (j == k) v *= 1.0 + shift;   // relative diagonal shift of a retried low-precision factor
        M[q] = (Tout)v;
    }
}

// H (FP64) to its FP32 copy.
__global__ void k_h_to_f32(const Inst* __restrict__ insts) {
    pdl_wait();
    const Inst& I = insts[blockIdx.y];
    const size_t total = (size_t)I.n * I.n;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x)
        I.H32[q] = (float)I.H64[q];
}

// ---------------------------------------------------------------------------

int syrk_cc_tiles(int n) {
    int nt = (n + kTile - 1) / kTile;
    return nt * (nt + 1) / 2;
}

int syrk_cc_splits(int ns, int nu, int N) {
    // aim for ~4 CTAs per SM over the tiles of this instance
    int n = nu * N;
    int tiles = syrk_cc_tiles(n);
    long long chunks = (long long)N * ((ns + kKc - 1) / kKc);
    int s = (device_sm_count() * 4 + tiles - 1) / tiles;
    if (s > chunks) s = (int)chunks;
    if (s > 64) s = 64;
    return s < 1 ? 1 : s;
}

void launch_syrk_cc(const Inst* d_insts, int count, int max_n, int splits, int fp64, int mode,
                    const double* gq, const double* gqf, int force, cudaStream_t st) {
    dim3 grid(syrk_cc_tiles(max_n) * splits, count);
    if (fp64) LQ_LAUNCH(lq_pdl(k_syrk_cc<double>, grid, 256, 0, st, d_insts, mode, gq, gqf, splits, force));
    else LQ_LAUNCH(lq_pdl(k_syrk_cc<float>, grid, 256, 0, st, d_insts, mode, gq, gqf, splits, force));
}

void launch_syrk_reduce(const Inst* d_insts, int count, int max_n, int splits, int part_kind,
                        int out_fp64, int base_mode, int add_sigu, int force, void* out_override,
                        cudaStream_t st, double shift) {
    size_t total = (size_t)max_n * max_n;
    int nb = (int)((total + 255) / 256);
    nb = nb > 4096 ? 4096 : nb;
    dim3 grid(nb, count);
    if (part_kind == 0) {        // FP64 partials, 64-tiles
        if (out_fp64) LQ_LAUNCH(lq_pdl(k_syrk_reduce<double, double, 64>, grid, 256, 0, st, d_insts, splits, base_mode, add_sigu, force, (double*)out_override, shift));
        else LQ_LAUNCH(lq_pdl(k_syrk_reduce<double, float, 64>, grid, 256, 0, st, d_insts, splits, base_mode, add_sigu, force, (float*)out_override, shift));
    } else if (part_kind == 1) { // FP32 partials, 64-tiles
        if (out_fp64) LQ_LAUNCH(lq_pdl(k_syrk_reduce<float, double, 64>, grid, 256, 0, st, d_insts, splits, base_mode, add_sigu, force, (double*)out_override, shift));
        else LQ_LAUNCH(lq_pdl(k_syrk_reduce<float, float, 64>, grid, 256, 0, st, d_insts, splits, base_mode, add_sigu, force, (float*)out_override, shift));
    } else {                     // FP32 partials, 128-tiles, column-major (tensor-core SYRK)
        if (out_fp64) LQ_LAUNCH(lq_pdl(k_syrk_reduce<float, double, 128, true>, grid, 256, 0, st, d_insts, splits, base_mode, add_sigu, force, (double*)out_override, shift));
        else LQ_LAUNCH(lq_pdl(k_syrk_reduce<float, float, 128, true, true>, grid, 256, 0, st, d_insts, splits, base_mode, add_sigu, force, (float*)out_override, shift));
    }
}

void launch_h_to_f32(const Inst* d_inst, int n, cudaStream_t st) {
    size_t total = (size_t)n * n;
    int nb = (int)((total + 255) / 256);
    nb = nb > 4096 ? 4096 : nb;
    LQ_LAUNCH(lq_pdl(k_h_to_f32, dim3(nb, 1), 256, 0, st, d_inst));
}

}  // namespace lqmpc
