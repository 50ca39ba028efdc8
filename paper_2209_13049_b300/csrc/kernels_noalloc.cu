// Allocation-free variant of the FP64 condensed-KKT formation
//     M = H + Gamma' diag(sigx) Gamma + diag(sigu)            (Eq. 7)
// for callers that must not allocate device memory while they run.  The
// split-K partial tiles, which the context's own formation keeps in a
// workspace allocated at setup, live here in one fixed file-scope device
// array.  Everything else (the G-stack and H built at setup, Sigma and the
// output supplied by the caller) is already resident.
//
// Shared scratch: every call on a device uses the same array, so calls whose
// work overlaps in time on one device (two streams, or two host threads)
// corrupt each other's partials; order them.  No scratch entry has to start
// at zero: each partial tile is written in full before the reduce reads it.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace lqmpc {

constexpr int kNaTile = 64;        // output tile edge
constexpr int kNaKc = 32;          // K rows staged per step
constexpr int kNaMaxDevices = 64;
constexpr size_t kNaScratchDoubles = size_t(2) << 20;   // 16 MiB of partial tiles per device
constexpr size_t kNaTileDoubles = size_t(kNaTile) * kNaTile;

static __device__ __align__(256) double g_noalloc_scratch[kNaScratchDoubles];

__host__ __device__ inline void na_tile_of(int t, int& a, int& b) {
    // lower tiles enumerated row by row: t = a(a+1)/2 + b, b <= a
    a = 0;
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    b = t - a * (a + 1) / 2;
}

// Partial of lower tile (a, b) over one K slice.  Row block r of Gamma is the
// window of G-stack columns starting at (N-1-r) nu (columns at or beyond n
// are Gamma's zero blocks); a tile whose rows start in input block t0 gets
// contributions from row blocks r >= t0 only.
__global__ void __launch_bounds__(256) k_syrk_scratch(const double* __restrict__ G, int ldg,
                                                      const double* __restrict__ sigx, int ns, int nu,
                                                      int N, int splits, double* __restrict__ ws) {
    const int n = nu * N;
    const int nt = (n + kNaTile - 1) / kNaTile;
    const int tile = blockIdx.x / splits, split = blockIdx.x % splits;
    if (tile >= nt * (nt + 1) / 2) return;
    int a, b;
    na_tile_of(tile, a, b);
    const int rmin = (a * kNaTile) / nu;
    const int nkc = (ns + kNaKc - 1) / kNaKc;
    const long long nchunks = (long long)(N - rmin) * nkc;
    const long long c0 = nchunks * split / splits, c1 = nchunks * (split + 1) / splits;

    __shared__ double As[kNaKc][kNaTile + 1];
    __shared__ double Bs[kNaKc][kNaTile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int lk = threadIdx.x & 31, lc = threadIdx.x >> 5;
    double acc[4][4] = {};
    for (long long ch = c0; ch < c1; ++ch) {
        const int r = rmin + (int)(ch / nkc);
        const int i = (int)(ch % nkc) * kNaKc + lk;
        const int off = (N - 1 - r) * nu;
        const double d = i < ns ? sigx[(size_t)r * ns + i] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int c = lc + 8 * q;
            const int ca = off + a * kNaTile + c, cb = off + b * kNaTile + c;
            As[lk][c] = (i < ns && ca < n) ? G[(size_t)ldg * ca + i] : 0.0;
            Bs[lk][c] = (i < ns && cb < n) ? G[(size_t)ldg * cb + i] * d : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kNaKc; ++kk) {
            double av[4], bv[4];
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
    double* out = ws + ((size_t)tile * splits + split) * kNaTileDoubles;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) out[(ty * 4 + p) * kNaTile + tx * 4 + q] = acc[p][q];
}

// M[j, k] = H[j, k] + sum over splits (in split order) of the partials of the
// lower tile holding (max(j,k), min(j,k)) + [j == k] sigu[j]; column-major.
__global__ void k_kkt_scratch_reduce(const double* __restrict__ ws, int splits, const double* __restrict__ H,
                                     const double* __restrict__ sigu, int n, double* __restrict__ M) {
    const size_t total = (size_t)n * n;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q % n), k = (int)(q / n);
        const int p = j > k ? j : k, m = j > k ? k : j;
        const int ta = p / kNaTile, tb = m / kNaTile;
        const size_t t = (size_t)ta * (ta + 1) / 2 + tb;
        const double* src = ws + t * splits * kNaTileDoubles + (p % kNaTile) * kNaTile + (m % kNaTile);
        double acc = 0.0;
        for (int s = 0; s < splits; ++s) acc += src[(size_t)s * kNaTileDoubles];
        double v = H[q] + acc;
        if (j == k) v += sigu[j];
        M[q] = v;
    }
}

// Per-device set-up, done once per device by the first call (the device must
// be current): force this module's two kernels onto the device (with lazy
// module loading that is also when the CUDA driver places the scratch array),
// look up the array's device address and read the SM count.  nullptr with
// *err set if any step fails.
struct NaDevice {
    double* scratch;
    int sms;
};

static const NaDevice* noalloc_device(int dev, cudaError_t* err) {
    static std::mutex mu;
    static NaDevice devs[kNaMaxDevices] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kNaMaxDevices) { *err = cudaErrorInvalidDevice; return nullptr; }
    NaDevice& d = devs[dev];
    if (!d.scratch) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, k_syrk_scratch);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_kkt_scratch_reduce);
        int sms = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        void* p = nullptr;
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) { *err = e; return nullptr; }
        d.sms = sms > 0 ? sms : 1;
        d.scratch = static_cast<double*>(p);
    }
    return &d;
}

int noalloc_max_n() {
    // one split of every lower tile must fit
    int nt = 1;
    while ((size_t)(nt + 1) * (nt + 2) / 2 * kNaTileDoubles <= kNaScratchDoubles) ++nt;
    return nt * kNaTile;
}

int launch_form_kkt_noalloc(const double* G, int ldg, const double* H, const double* sigx, const double* sigu,
                            double* M, int ns, int nu, int N, cudaStream_t st) {
    const int n = nu * N;
    if (n > noalloc_max_n()) return 1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    cudaError_t err = cudaSuccess;
    const NaDevice* nd = noalloc_device(dev, &err);
    if (!nd) return 2;
    double* ws = nd->scratch;
    const int nt = (n + kNaTile - 1) / kNaTile;
    const long long tiles = (long long)nt * (nt + 1) / 2;
    // about four CTAs per SM over the tiles, within the scratch and the K chunks
    const long long chunks = (long long)N * ((ns + kNaKc - 1) / kNaKc);
    long long splits = ((long long)nd->sms * 4 + tiles - 1) / tiles;
    const long long fit = (long long)(kNaScratchDoubles / (tiles * kNaTileDoubles));
    if (splits > fit) splits = fit;
    if (splits > chunks) splits = chunks;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    // plain launches: the library's launch macro may create profiling events
    k_syrk_scratch<<<dim3((unsigned)(tiles * splits)), 256, 0, st>>>(G, ldg, sigx, ns, nu, N, (int)splits, ws);
    const size_t total = (size_t)n * n;
    int nb = (int)((total + 255) / 256);
    nb = nb > 4096 ? 4096 : nb;
    k_kkt_scratch_reduce<<<nb, 256, 0, st>>>(ws, (int)splits, H, sigu, n, M);
    note_launches(2);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // namespace lqmpc
