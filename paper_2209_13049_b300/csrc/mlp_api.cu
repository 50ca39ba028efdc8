// C ABI of the warm-start network (lqmpc_mlp_*): device buffers, tensor
// maps and the launch sequences of one training step and of inference.
// Layout (all row-major; P = padded):
//   W1 nh x inP, W2 nh x nh, W3 outP x nh (FP32 master, BF16 W and W^T),
//   activations Bmax x width (BF16) with transposed copies width x Bmax,
//   pre-activations Z1, Z2 and the output Y3 in FP32.
// inP, nh, outP and Bmax are multiples of 128; padding rows and columns of
// the weights start at zero and stay zero (their gradients are zero).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "lqmpc.h"

using namespace lqmpc;

#define CK_RET(x)                                        \
    do {                                                 \
        if ((x) != cudaSuccess) return LQMPC_ERR_CUDA;   \
    } while (0)

namespace {

int round_up(int v, int a) { return (v + a - 1) / a * a; }

// splitmix64: seeded, platform-independent initial weights and shuffles
struct SplitMix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

struct Map {
    alignas(64) unsigned char b[128];
};

}  // namespace

struct lqmpc_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nin = 0, nh = 0, nout = 0, inP = 0, outP = 0, Bmax = 0;
    size_t nparam = 0;                 // FP32 parameters, padded layout
    void* arena = nullptr;
    // parameters (views into one FP32 block): W1 b1 W2 b2 W3 b3
    float *prm = nullptr, *grd = nullptr, *mom = nullptr, *vel = nullptr;
    size_t off[6] = {}, cnt[6] = {};
    int rows[6] = {}, cols[6] = {};
    __nv_bfloat16 *Wb[3] = {}, *Wt[3] = {};
    __nv_bfloat16 *X = nullptr, *XT = nullptr, *Y1 = nullptr, *Y1T = nullptr, *Y2 = nullptr, *Y2T = nullptr;
    __nv_bfloat16 *G3 = nullptr, *G3T = nullptr, *G2 = nullptr, *G2T = nullptr, *G1 = nullptr, *G1T = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Y3 = nullptr, *T = nullptr;
    double *lo = nullptr, *hi = nullptr, *loss_part = nullptr, *loss = nullptr, *xin = nullptr, *uout = nullptr;
    int *idx = nullptr, *err = nullptr, *tstep = nullptr;
    double* h_loss = nullptr;          // pinned
    Map mX, mXT, mW[3], mWT[3], mY1, mY1T, mY2, mY2T, mG3, mG3T, mG2, mG2T, mG1T;
    int step_kernels = 0;              // kernel launches of one captured training step
};

namespace {

float* P(lqmpc_mlp* m, float* base, int k) { return base + m->off[k]; }

// Forward pass over Bp rows (multiple of 128); the last layer either forms
// the loss and its gradient (train) or projects onto [lo, hi] (inference).
void forward(lqmpc_mlp* m, int Bp, int B, bool train) {
    cudaStream_t st = m->stream;
    GemmEpi e{};
    e.err = m->err;
    e.ldt = m->Bmax;
    e.m_real = B;
    // layer 1: X (Bp x inP) W1^T -> Z1, Y1, Y1^T
    e.M = Bp; e.N = m->nh; e.bias = P(m, m->prm, 1); e.zf = m->Z1; e.yb = m->Y1; e.ybt = m->Y1T;
    mlp_gemm(EPI_BIAS_GELU, m->mX.b, m->mW[0].b, Bp, m->nh, m->inP, e, st);
    // layer 2
    e.bias = P(m, m->prm, 3); e.zf = m->Z2; e.yb = m->Y2; e.ybt = m->Y2T;
    mlp_gemm(EPI_BIAS_GELU, m->mY1.b, m->mW[1].b, Bp, m->nh, m->nh, e, st);
    // layer 3
    e.N = m->outP; e.bias = P(m, m->prm, 5);
    if (train) {
        e.zf = m->Y3; e.yb = m->G3; e.ybt = m->G3T; e.target = m->T; e.n_real = m->nout;
        e.gscale = 2.0f / ((float)B * (float)m->nout);
        e.loss_part = m->loss_part;
        mlp_gemm(EPI_BIAS_LOSS, m->mY2.b, m->mW[2].b, Bp, m->outP, m->nh, e, st);
        mlp_sum(m->loss_part, (Bp / 128) * (m->outP / 128), m->loss, st);
    } else {
        e.n_real = m->nout; e.lo = m->lo; e.hi = m->hi; e.out64 = m->uout;
        mlp_gemm(EPI_BIAS_PROJ, m->mY2.b, m->mW[2].b, Bp, m->outP, m->nh, e, st);
    }
}

// Backward pass (gradients into grd); assumes forward(train) ran on the same rows.
void backward(lqmpc_mlp* m, int Bp) {
    cudaStream_t st = m->stream;
    GemmEpi e{};
    e.err = m->err;
    e.ldt = m->Bmax;
    // dW3 = G3^T Y2 (outP x nh), K = Bp
    e.M = m->outP; e.N = m->nh; e.zf = P(m, m->grd, 4);
    mlp_gemm(EPI_WGRAD, m->mG3T.b, m->mY2T.b, m->outP, m->nh, Bp, e, st);
    mlp_colsum(m->G3T, m->outP, Bp, m->Bmax, P(m, m->grd, 5), st);
    // dY2 = G3 W3 -> G2 = dY2 * GELU'(Z2), K = outP
    e.M = Bp; e.N = m->nh; e.zin = m->Z2; e.yb = m->G2; e.ybt = m->G2T;
    mlp_gemm(EPI_GELU_BWD, m->mG3.b, m->mWT[2].b, Bp, m->nh, m->outP, e, st);
    // dW2 = G2^T Y1
    e.M = m->nh; e.N = m->nh; e.zf = P(m, m->grd, 2);
    mlp_gemm(EPI_WGRAD, m->mG2T.b, m->mY1T.b, m->nh, m->nh, Bp, e, st);
    mlp_colsum(m->G2T, m->nh, Bp, m->Bmax, P(m, m->grd, 3), st);
    // dY1 = G2 W2 -> G1
    e.M = Bp; e.N = m->nh; e.zin = m->Z1; e.yb = m->G1; e.ybt = m->G1T;
    mlp_gemm(EPI_GELU_BWD, m->mG2.b, m->mWT[1].b, Bp, m->nh, m->nh, e, st);
    // dW1 = G1^T X
    e.M = m->nh; e.N = m->inP; e.zf = P(m, m->grd, 0);
    mlp_gemm(EPI_WGRAD, m->mG1T.b, m->mXT.b, m->nh, m->inP, Bp, e, st);
    mlp_colsum(m->G1T, m->nh, Bp, m->Bmax, P(m, m->grd, 1), st);
}

void adam(lqmpc_mlp* m, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    mlp_tick(m->tstep, m->stream);
    for (int k = 0; k < 6; ++k) {
        const bool wmat = (k % 2) == 0;
        mlp_adam(P(m, m->prm, k), P(m, m->grd, k), P(m, m->mom, k), P(m, m->vel, k), m->cnt[k], lr, b1, b2, eps,
                 m->tstep, m->rows[k], m->cols[k], wmat ? m->Wb[k / 2] : nullptr, wmat ? m->Wt[k / 2] : nullptr,
                 m->stream);
    }
}

lqmpc_status sync_err(lqmpc_mlp* m) {
    int err = 0;
    if (cudaMemcpyAsync(&err, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess) return LQMPC_ERR_CUDA;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return LQMPC_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return LQMPC_ERR_CUDA;
    return err ? LQMPC_ERR_TIMEOUT : LQMPC_OK;
}

// Logical (unpadded) <-> padded parameter layout.
void to_padded(const lqmpc_mlp* m, const float* logical, std::vector<float>& padded) {
    padded.assign(m->nparam, 0.0f);
    const int lr[6] = {m->nh, m->nh, m->nh, m->nh, m->nout, m->nout};
    const int lc[6] = {m->nin, 1, m->nh, 1, m->nh, 1};
    size_t q = 0;
    for (int k = 0; k < 6; ++k)
        for (int r = 0; r < lr[k]; ++r)
            for (int c = 0; c < lc[k]; ++c) padded[m->off[k] + (size_t)r * m->cols[k] + c] = logical[q++];
}

void to_logical(const lqmpc_mlp* m, const std::vector<float>& padded, float* logical) {
    const int lr[6] = {m->nh, m->nh, m->nh, m->nh, m->nout, m->nout};
    const int lc[6] = {m->nin, 1, m->nh, 1, m->nh, 1};
    size_t q = 0;
    for (int k = 0; k < 6; ++k)
        for (int r = 0; r < lr[k]; ++r)
            for (int c = 0; c < lc[k]; ++c) logical[q++] = padded[m->off[k] + (size_t)r * m->cols[k] + c];
}

lqmpc_status upload_params(lqmpc_mlp* m, const std::vector<float>& padded) {
    if (cudaMemcpyAsync(m->prm, padded.data(), sizeof(float) * m->nparam, cudaMemcpyHostToDevice, m->stream) !=
        cudaSuccess)
        return LQMPC_ERR_CUDA;
    cudaMemsetAsync(m->mom, 0, sizeof(float) * m->nparam, m->stream);
    cudaMemsetAsync(m->vel, 0, sizeof(float) * m->nparam, m->stream);
    cudaMemsetAsync(m->tstep, 0, sizeof(int), m->stream);
    for (int k = 0; k < 3; ++k) mlp_cast(P(m, m->prm, 2 * k), m->rows[2 * k], m->cols[2 * k], m->Wb[k], m->Wt[k], m->stream);
    return sync_err(m);
}

}  // namespace

extern "C" {

lqmpc_status lqmpc_mlp_create(lqmpc_mlp** out, int n_in, int n_hidden, int n_out, int max_batch,
                              unsigned long long seed, void* stream) {
    if (!out) return LQMPC_ERR_ARG;
    *out = nullptr;
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1 || n_hidden % 128 != 0 || n_in > (1 << 16) ||
        n_out > (1 << 16) || n_hidden > 8192 || max_batch > (1 << 16))
        return LQMPC_ERR_ARG;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) return LQMPC_ERR_CUDA;
    lqmpc_mlp* m = new (std::nothrow) lqmpc_mlp();
    if (!m) return LQMPC_ERR_CUDA;
    cudaGetDevice(&m->device);
    m->stream = (cudaStream_t)stream;
    if (!stream) {
        if (cudaStreamCreate(&m->stream) != cudaSuccess) { delete m; return LQMPC_ERR_CUDA; }
        m->own_stream = true;
    }
    m->nin = n_in; m->nh = n_hidden; m->nout = n_out;
    m->inP = round_up(n_in, 128); m->outP = round_up(n_out, 128); m->Bmax = round_up(max_batch, 128);
    const int rows[6] = {m->nh, m->nh, m->nh, m->nh, m->outP, m->outP};
    const int cols[6] = {m->inP, 1, m->nh, 1, m->nh, 1};
    size_t o = 0;
    for (int k = 0; k < 6; ++k) {
        m->rows[k] = rows[k]; m->cols[k] = cols[k];
        m->off[k] = o; m->cnt[k] = (size_t)rows[k] * cols[k];
        o += (m->cnt[k] + 63) / 64 * 64;
    }
    m->nparam = o;
    // one arena, 256-byte aligned pieces
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t at = bytes; bytes += (b + 255) / 256 * 256; return at; };
    const size_t B = m->Bmax, IN = m->inP, H = m->nh, OUT = m->outP, bf = sizeof(__nv_bfloat16);
    size_t a_prm = take(4 * o), a_grd = take(4 * o), a_mom = take(4 * o), a_vel = take(4 * o);
    size_t a_wb[3], a_wt[3];
    for (int k = 0; k < 3; ++k) { a_wb[k] = take(bf * m->cnt[2 * k]); a_wt[k] = take(bf * m->cnt[2 * k]); }
    size_t a_X = take(bf * B * IN), a_XT = take(bf * B * IN), a_Y1 = take(bf * B * H), a_Y1T = take(bf * B * H);
    size_t a_Y2 = take(bf * B * H), a_Y2T = take(bf * B * H), a_G3 = take(bf * B * OUT), a_G3T = take(bf * B * OUT);
    size_t a_G2 = take(bf * B * H), a_G2T = take(bf * B * H), a_G1 = take(bf * B * H), a_G1T = take(bf * B * H);
    size_t a_Z1 = take(4 * B * H), a_Z2 = take(4 * B * H), a_Y3 = take(4 * B * OUT), a_T = take(4 * B * OUT);
    size_t a_lo = take(8 * OUT), a_hi = take(8 * OUT), a_lp = take(8 * (B / 128) * (OUT / 128)), a_loss = take(8);
    size_t a_xin = take(8 * B * (size_t)n_in), a_uout = take(8 * B * (size_t)n_out);
    size_t a_idx = take(4 * B), a_err = take(4), a_t = take(4);
    if (cudaMalloc(&m->arena, bytes) != cudaSuccess) { lqmpc_mlp_free(m); return LQMPC_ERR_CUDA; }
    unsigned char* base = (unsigned char*)m->arena;
    cudaMemsetAsync(base, 0, bytes, m->stream);
    m->prm = (float*)(base + a_prm); m->grd = (float*)(base + a_grd); m->mom = (float*)(base + a_mom);
    m->vel = (float*)(base + a_vel);
    for (int k = 0; k < 3; ++k) { m->Wb[k] = (__nv_bfloat16*)(base + a_wb[k]); m->Wt[k] = (__nv_bfloat16*)(base + a_wt[k]); }
    m->X = (__nv_bfloat16*)(base + a_X); m->XT = (__nv_bfloat16*)(base + a_XT);
    m->Y1 = (__nv_bfloat16*)(base + a_Y1); m->Y1T = (__nv_bfloat16*)(base + a_Y1T);
    m->Y2 = (__nv_bfloat16*)(base + a_Y2); m->Y2T = (__nv_bfloat16*)(base + a_Y2T);
    m->G3 = (__nv_bfloat16*)(base + a_G3); m->G3T = (__nv_bfloat16*)(base + a_G3T);
    m->G2 = (__nv_bfloat16*)(base + a_G2); m->G2T = (__nv_bfloat16*)(base + a_G2T);
    m->G1 = (__nv_bfloat16*)(base + a_G1); m->G1T = (__nv_bfloat16*)(base + a_G1T);
    m->Z1 = (float*)(base + a_Z1); m->Z2 = (float*)(base + a_Z2); m->Y3 = (float*)(base + a_Y3); m->T = (float*)(base + a_T);
    m->lo = (double*)(base + a_lo); m->hi = (double*)(base + a_hi); m->loss_part = (double*)(base + a_lp);
    m->loss = (double*)(base + a_loss); m->xin = (double*)(base + a_xin); m->uout = (double*)(base + a_uout);
    m->idx = (int*)(base + a_idx); m->err = (int*)(base + a_err); m->tstep = (int*)(base + a_t);
    if (cudaMallocHost(&m->h_loss, sizeof(double)) != cudaSuccess) { lqmpc_mlp_free(m); return LQMPC_ERR_CUDA; }
    // tensor maps: A operands (rows x K) and B operands (N x K), all K-major BF16
    bool ok = mlp_make_map(m->mX.b, m->X, (int)B, (int)IN) && mlp_make_map(m->mXT.b, m->XT, (int)IN, (int)B) &&
              mlp_make_map(m->mY1.b, m->Y1, (int)B, (int)H) && mlp_make_map(m->mY1T.b, m->Y1T, (int)H, (int)B) &&
              mlp_make_map(m->mY2.b, m->Y2, (int)B, (int)H) && mlp_make_map(m->mY2T.b, m->Y2T, (int)H, (int)B) &&
              mlp_make_map(m->mG3.b, m->G3, (int)B, (int)OUT) && mlp_make_map(m->mG3T.b, m->G3T, (int)OUT, (int)B) &&
              mlp_make_map(m->mG2.b, m->G2, (int)B, (int)H) && mlp_make_map(m->mG2T.b, m->G2T, (int)H, (int)B) &&
              mlp_make_map(m->mG1T.b, m->G1T, (int)H, (int)B);
    for (int k = 0; k < 3 && ok; ++k)
        ok = mlp_make_map(m->mW[k].b, m->Wb[k], m->rows[2 * k], m->cols[2 * k]) &&
             mlp_make_map(m->mWT[k].b, m->Wt[k], m->cols[2 * k], m->rows[2 * k]);
    if (!ok) { lqmpc_mlp_free(m); return LQMPC_ERR_UNSUPPORTED; }
    // initial weights and biases ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) on the real rows/columns
    std::vector<float> logical((size_t)n_hidden * n_in + n_hidden + (size_t)n_hidden * n_hidden + n_hidden +
                               (size_t)n_out * n_hidden + n_out);
    SplitMix rng{seed};
    const int fan[6] = {n_in, n_in, n_hidden, n_hidden, n_hidden, n_hidden};
    const size_t len[6] = {(size_t)n_hidden * n_in, (size_t)n_hidden, (size_t)n_hidden * n_hidden, (size_t)n_hidden,
                           (size_t)n_out * n_hidden, (size_t)n_out};
    size_t q = 0;
    for (int k = 0; k < 6; ++k) {
        const double a = 1.0 / std::sqrt((double)fan[k]);
        for (size_t i = 0; i < len[k]; ++i) logical[q++] = (float)((2.0 * rng.uniform() - 1.0) * a);
    }
    std::vector<float> padded;
    to_padded(m, logical.data(), padded);
    std::vector<double> lo(m->outP, -INFINITY), hi(m->outP, INFINITY);
    cudaMemcpyAsync(m->lo, lo.data(), 8 * lo.size(), cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->hi, hi.data(), 8 * hi.size(), cudaMemcpyHostToDevice, m->stream);
    lqmpc_status s = upload_params(m, padded);
    if (s != LQMPC_OK) { lqmpc_mlp_free(m); return s; }
    *out = m;
    return LQMPC_OK;
}

void lqmpc_mlp_free(lqmpc_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    cudaFree(m->arena);
    if (m->h_loss) cudaFreeHost(m->h_loss);
    if (m->own_stream) cudaStreamDestroy(m->stream);
    delete m;
}

lqmpc_status lqmpc_mlp_set_bounds(lqmpc_mlp* m, const double* lo, const double* hi) {
    if (!m || !lo || !hi) return LQMPC_ERR_ARG;
    for (int j = 0; j < m->nout; ++j)
        if (std::isnan(lo[j]) || std::isnan(hi[j]) || lo[j] > hi[j]) return LQMPC_ERR_ARG;
    CK_RET(cudaSetDevice(m->device));
    CK_RET(cudaMemcpyAsync(m->lo, lo, 8 * (size_t)m->nout, cudaMemcpyHostToDevice, m->stream));
    CK_RET(cudaMemcpyAsync(m->hi, hi, 8 * (size_t)m->nout, cudaMemcpyHostToDevice, m->stream));
    CK_RET(cudaStreamSynchronize(m->stream));
    return LQMPC_OK;
}

lqmpc_status lqmpc_mlp_get_params(lqmpc_mlp* m, float* params) {
    if (!m || !params) return LQMPC_ERR_ARG;
    CK_RET(cudaSetDevice(m->device));
    std::vector<float> padded(m->nparam);
    CK_RET(cudaMemcpyAsync(padded.data(), m->prm, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, m->stream));
    CK_RET(cudaStreamSynchronize(m->stream));
    to_logical(m, padded, params);
    return LQMPC_OK;
}

lqmpc_status lqmpc_mlp_set_params(lqmpc_mlp* m, const float* params) {
    if (!m || !params) return LQMPC_ERR_ARG;
    CK_RET(cudaSetDevice(m->device));
    std::vector<float> padded;
    to_padded(m, params, padded);
    for (float v : padded)
        if (!std::isfinite(v)) return LQMPC_ERR_ARG;
    return upload_params(m, padded);
}

lqmpc_status lqmpc_mlp_grad(lqmpc_mlp* m, const float* X, const float* U, int B, float* grads, double* loss) {
    if (!m || !X || !U || !grads || B < 1 || B > m->Bmax) return LQMPC_ERR_ARG;
    CK_RET(cudaSetDevice(m->device));
    const int Bp = round_up(B, 128);
    float *dx = nullptr, *du = nullptr;
    int* didx = nullptr;
    if (cudaMalloc(&dx, sizeof(float) * (size_t)B * m->nin) != cudaSuccess ||
        cudaMalloc(&du, sizeof(float) * (size_t)B * m->nout) != cudaSuccess ||
        cudaMalloc(&didx, sizeof(int) * (size_t)B) != cudaSuccess) {
        cudaFree(dx); cudaFree(du); cudaFree(didx);
        return LQMPC_ERR_CUDA;
    }
    std::vector<int> id(B);
    for (int i = 0; i < B; ++i) id[i] = i;
    lqmpc_status s = LQMPC_OK;
    if (cudaMemcpyAsync(dx, X, sizeof(float) * (size_t)B * m->nin, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(du, U, sizeof(float) * (size_t)B * m->nout, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(didx, id.data(), sizeof(int) * B, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        s = LQMPC_ERR_CUDA;
    if (s == LQMPC_OK) {
        cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
        mlp_gather(dx, du, didx, B, Bp, m->Bmax, m->nin, m->inP, m->nout, m->outP, m->X, m->XT, m->T, m->stream);
        forward(m, Bp, B, true);
        backward(m, Bp);
        s = sync_err(m);
    }
    if (s == LQMPC_OK) {
        std::vector<float> padded(m->nparam);
        double l = 0.0;
        if (cudaMemcpy(padded.data(), m->grd, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            s = LQMPC_ERR_CUDA;
        else {
            to_logical(m, padded, grads);
            if (loss) *loss = l / ((double)B * m->nout);
        }
    }
    cudaFree(dx); cudaFree(du); cudaFree(didx);
    return s;
}

lqmpc_status lqmpc_mlp_train(lqmpc_mlp* m, const float* X, const float* U, int S, int epochs, int batch, float lr,
                             unsigned long long seed, double* epoch_loss) {
    if (!m || !X || !U || S < 1 || epochs < 0 || batch < 1 || batch > m->Bmax || batch > S || !(lr > 0.0f))
        return LQMPC_ERR_ARG;
    CK_RET(cudaSetDevice(m->device));
    const int Bp = round_up(batch, 128);
    const int steps = S / batch;
    float *dx = nullptr, *du = nullptr;
    int* perm = nullptr;
    if (cudaMalloc(&dx, sizeof(float) * (size_t)S * m->nin) != cudaSuccess ||
        cudaMalloc(&du, sizeof(float) * (size_t)S * m->nout) != cudaSuccess ||
        cudaMalloc(&perm, sizeof(int) * (size_t)S) != cudaSuccess) {
        cudaFree(dx); cudaFree(du); cudaFree(perm);
        return LQMPC_ERR_CUDA;
    }
    lqmpc_status s = LQMPC_OK;
    if (cudaMemcpyAsync(dx, X, sizeof(float) * (size_t)S * m->nin, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(du, U, sizeof(float) * (size_t)S * m->nout, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        s = LQMPC_ERR_CUDA;
    std::vector<int> p(S);
    SplitMix rng{seed};
    // one training step (gather -> forward -> backward -> Adam), captured once
    cudaGraphExec_t exec = nullptr;
    auto step_body = [&]() {
        mlp_gather(dx, du, m->idx, batch, Bp, m->Bmax, m->nin, m->inP, m->nout, m->outP, m->X, m->XT, m->T, m->stream);
        forward(m, Bp, batch, true);
        backward(m, Bp);
        adam(m, lr);
    };
    const char* ge = getenv("LQMPC_GRAPH");
    bool use_graph = !(ge && ge[0] == '0');
    for (int ep = 0; ep < epochs && s == LQMPC_OK; ++ep) {
        for (int i = 0; i < S; ++i) p[i] = i;
        for (int i = S - 1; i > 0; --i) {          // Fisher-Yates
            const int j = (int)(rng.next() % (uint64_t)(i + 1));
            std::swap(p[i], p[j]);
        }
        if (cudaMemcpyAsync(perm, p.data(), sizeof(int) * (size_t)S, cudaMemcpyHostToDevice, m->stream) != cudaSuccess) {
            s = LQMPC_ERR_CUDA;
            break;
        }
        cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
        for (int k = 0; k < steps; ++k) {
            cudaMemcpyAsync(m->idx, perm + (size_t)k * batch, sizeof(int) * batch, cudaMemcpyDeviceToDevice, m->stream);
            if (use_graph && !exec) {
                cudaGraph_t g = nullptr;
                const unsigned long long k0 = lqmpc_kernel_launches();
                if (cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                    step_body();
                    const unsigned long long nk = lqmpc_kernel_launches() - k0;
                    note_launches(-(int)nk);
                    if (cudaStreamEndCapture(m->stream, &g) == cudaSuccess && g &&
                        cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
                        // replays count their kernels
                    } else {
                        exec = nullptr;
                        use_graph = false;
                        cudaGetLastError();
                    }
                    if (g) cudaGraphDestroy(g);
                    if (exec) m->step_kernels = (int)nk;
                } else {
                    use_graph = false;
                    cudaGetLastError();
                }
            }
            if (exec) {
                cudaGraphLaunch(exec, m->stream);
                note_launches(m->step_kernels);
            } else {
                step_body();
            }
        }
        s = sync_err(m);
        if (s == LQMPC_OK && epoch_loss) {
            double l = 0.0;
            if (cudaMemcpy(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) s = LQMPC_ERR_CUDA;
            epoch_loss[ep] = steps > 0 ? l / ((double)steps * batch * m->nout) : 0.0;
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaStreamSynchronize(m->stream);
    cudaFree(dx); cudaFree(du); cudaFree(perm);
    return s;
}

lqmpc_status lqmpc_mlp_infer(lqmpc_mlp* m, const double* x, int count, double* u_out) {
    if (!m || !x || !u_out || count < 1) return LQMPC_ERR_ARG;
    CK_RET(cudaSetDevice(m->device));
    for (int done = 0; done < count; done += m->Bmax) {
        const int c = count - done < m->Bmax ? count - done : m->Bmax;
        const int Bp = round_up(c, 128);
        CK_RET(cudaMemcpyAsync(m->xin, x + (size_t)done * m->nin, sizeof(double) * (size_t)c * m->nin,
                               cudaMemcpyHostToDevice, m->stream));
        mlp_load_x(m->xin, c, m->nin, m->inP, Bp, m->X, m->stream);
        forward(m, Bp, c, false);
        CK_RET(cudaMemcpyAsync(u_out + (size_t)done * m->nout, m->uout, sizeof(double) * (size_t)c * m->nout,
                               cudaMemcpyDeviceToHost, m->stream));
        lqmpc_status s = sync_err(m);
        if (s != LQMPC_OK) return s;
    }
    return LQMPC_OK;
}

}  // extern "C"
