// Host side of the lqmpc C ABI: context and device-arena management, the
// one-time setup (state elimination and H), and the interior-point driver.
//
// One solve is the paper's Algorithm 1 with Mehrotra's predictor-corrector
// step: per iteration
//   residuals and Sigma -> stop test -> form M = H + Gamma' Sigma_x Gamma +
//   Sigma_u -> Cholesky -> predictor solve -> affine step length and sigma ->
//   corrector right-hand side -> corrector solve -> step length -> update.
// Every launch covers a batch of instances (grid.y); a single solve is a
// batch of one.  The host waits on the device once per iteration (to learn
// whether every instance has finished) and, in the mixed-precision modes,
// once after each refined solve (to decide on the FP64 fallback).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lqmpc.h"
#include "common.cuh"
#include "kernels.h"

using namespace lqmpc;

#include <atomic>

namespace lqmpc {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }
static int g_prof = -1;
static std::vector<cudaEvent_t> g_prof_pool;
static size_t g_prof_next = 0;
struct ProfRec { const char* what; cudaEvent_t a, b; };
static std::vector<ProfRec> g_prof_recs;
static cudaEvent_t prof_event() {
    if (g_prof_next == g_prof_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_prof_pool.push_back(e);
    }
    return g_prof_pool[g_prof_next++];
}
cudaEvent_t prof_start(cudaStream_t st) {
    if (g_prof < 0) {
        const char* e = getenv("LQMPC_PROFILE");
        g_prof = (e && e[0] == '1') ? 1 : 0;
    }
    if (!g_prof) return nullptr;
    cudaEvent_t e = prof_event();
    cudaEventRecord(e, st);
    return e;
}
void prof_stop(cudaStream_t st, cudaEvent_t e0, const char* what) {
    if (!e0) return;
    cudaEvent_t e1 = prof_event();
    cudaEventRecord(e1, st);
    g_prof_recs.push_back({what, e0, e1});
}
// Print and clear the per-kernel table (kernel name = lq_pdl's first argument).
static void prof_report(const char* title) {
    if (g_prof != 1 || g_prof_recs.empty()) return;
    cudaDeviceSynchronize();
    struct Agg { std::string name; double ms; int n; };
    std::vector<Agg> aggs;
    double total = 0;
    for (auto& r : g_prof_recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        std::string nm(r.what);
        size_t k = nm.find("lq_pdl(");
        if (k != std::string::npos) {       // the kernel: lq_pdl's first argument
            nm = nm.substr(k + 7);
            int depth = 0;
            size_t e = 0;
            for (; e < nm.size(); ++e) {
                if (nm[e] == '<') ++depth;
                else if (nm[e] == '>') --depth;
                else if (nm[e] == ',' && depth == 0) break;
            }
            nm = nm.substr(0, e);
        }
        k = nm.find("<<<");
        if (k != std::string::npos) nm = nm.substr(0, k);
        bool found = false;
        for (auto& a : aggs)
            if (a.name == nm) { a.ms += ms; a.n++; found = true; break; }
        if (!found) aggs.push_back({nm, ms, 1});
        total += ms;
    }
    std::sort(aggs.begin(), aggs.end(), [](const Agg& x, const Agg& y) { return x.ms > y.ms; });
    fprintf(stderr, "lqmpc profile (%s): %.3f ms in %zu launches\n", title, total, g_prof_recs.size());
    for (auto& a : aggs)
        fprintf(stderr, "  %10.3f ms %5.1f%% %6d x %8.2f us  %s\n", a.ms, 100.0 * a.ms / total, a.n,
                1e3 * a.ms / a.n, a.name.c_str());
    g_prof_recs.clear();
    g_prof_next = 0;
}
static int g_check = -1;
void check_launch(cudaStream_t st, const char* what, const char* file, int line) {
    if (g_check < 0) {
        const char* e = getenv("LQMPC_CHECK");
        g_check = (e && e[0] == '1') ? 1 : 0;
    }
    if (!g_check) return;
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        fprintf(stderr, "lqmpc check: %s / %s after %s (%s:%d)\n", cudaGetErrorString(e1), cudaGetErrorString(e2),
                what, file, line);
        fflush(stderr);
    }
}
// Programmatic dependent launch of the library's kernels (LQMPC_PDL=0: off).
bool pdl_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("LQMPC_PDL");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

}  // namespace lqmpc

namespace lqmpc {
// Captured CUDA graphs of the fixed launch sequences of an iteration (keyed
// by segment and precision).  Every kernel reads its data through the
// instance descriptors in device memory, so a graph stays valid for as long
// as the descriptor array it was captured with.
struct GraphSeg {
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;   // kernel launches one replay performs (before any loop)
    unsigned long long pass_kernels = 0;   // kernel launches of one pass of its device-side loop
    bool bad = false;                 // capture or instantiation failed: launch directly
    int timer_bits = 0;               // an iteration graph: the SYRK / factor timers its launches record
};
struct GraphCache {
    std::map<int, GraphSeg> segs;
    ~GraphCache() {
        for (auto& kv : segs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    }
};
}  // namespace lqmpc

struct lqmpc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;       // where the context's work runs
    cudaStream_t user_stream = nullptr;  // the stream given at setup (NULL: legacy default)
    bool own_stream = false;             // stream created here for a NULL user stream
    lqmpc_options opts;
    Inst h;                     // host copy of the descriptor
    Inst* d_inst = nullptr;     // device copy
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    Scal* h_scal = nullptr;     // pinned host mirror of the Scal
    double* h_trace = nullptr;
    int trace_rows = 0;
    int cc_splits = 1;          // CUDA-core SYRK split-K factor
    int tc_splits = 1;          // tensor-core SYRK split-K factor
    int tc_ok = 0;              // tensor maps built
    void* d_maps = nullptr;     // 3 CUtensorMap (BF16, TF32, TF32 low part), 64-byte aligned, device
    cudaEvent_t ev[4];
    cudaEvent_t ev_read = nullptr;   // end of the copy of the instance state to the host
    cudaEvent_t evk[6];         // around the SYRK launch (tensor-core pair, CUDA-core pair) and the FP32 factor
    bool events = false;
    // per-solve SYRK timing
    double t_tc = 0, t_cc = 0, t_cc64 = 0, t_tc3 = 0, t_pf = 0;
    int n_tc = 0, n_cc = 0, n_cc64 = 0, n_tc3 = 0, n_pf = 0;
    lqmpc::GraphCache* graphs = nullptr;   // single-instance solves (d_inst is fixed)
    bool lyap = false;                     // FP64 KKT matrix by the Horner chains (sparse A)
    // side stream: the residual head's Gamma' product and r_d run there while
    // the context's stream forms and factors M (joined before the solves)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // general data (lqmpc_setup_general): device copies of S and w, and with a
    // feedback K the row of the lifted state that holds u_t (-1: u is the
    // solver's own variable)
    double* gen_dev = nullptr;
    int u_row = -1;
    // the caller's state dimension (x0 holds this many values); the lifted
    // rows of lqmpc_setup_general come after it and start at zero
    int ns_plant = 0;
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
    unsigned char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool all_finite(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

bool csr_ok(int n, const int* ptr, const int* idx, const double* val) {
    if (!ptr || (!idx && ptr[n] > 0) || (!val && ptr[n] > 0) || ptr[0] != 0) return false;
    for (int r = 0; r < n; ++r)
        if (ptr[r + 1] < ptr[r]) return false;
    for (int k = 0; k < ptr[n]; ++k)
        if (idx[k] < 0 || idx[k] >= n || !std::isfinite(val[k])) return false;
    return true;
}

bool csr_diag(int n, const int* ptr, const int* idx, const double* val, std::vector<double>& d) {
    d.assign(n, 0.0);
    for (int r = 0; r < n; ++r)
        for (int k = ptr[r]; k < ptr[r + 1]; ++k) {
            if (idx[k] != r) {
                if (val[k] != 0.0) return false;
            } else {
                d[r] += val[k];
            }
        }
    return true;
}

#define CK(x)                                                                        \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) {                                                     \
            if (getenv("LQMPC_DEBUG"))                                               \
                fprintf(stderr, "lqmpc: %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return LQMPC_ERR_CUDA;                                                   \
        }                                                                            \
    } while (0)

// Lay out every device array of an instance in one arena.
template <bool kAssign>
size_t layout(Inst& I, unsigned char* base, int nnzA, int nnzQ, int nnzQf, int max_iter,
              int cc_splits, int tc_splits, int nnzB, bool /*lyap: no buffers of its own*/) {
    Carver c{base};
    const int ns = I.ns, nu = I.nu, n = I.n, SX = I.SX;
    const size_t G = (size_t)I.ldg * n;
    auto at_ptr = c.take<int>(ns + 1); auto at_idx = c.take<int>(nnzA); auto at_val = c.take<double>(nnzA);
    auto bc_ptr = c.take<int>(nu + 1); auto bc_idx = c.take<int>(nnzB); auto bc_val = c.take<double>(nnzB);
    auto at_pack = c.take<int>(4 * (size_t)nnzA); auto bc_ff = c.take<float>(2 * (size_t)nnzB);
    auto sig_ff = c.take<float>(2 * (size_t)I.SX);
    auto a_ptr = c.take<int>(ns + 1); auto a_idx = c.take<int>(nnzA); auto a_val = c.take<double>(nnzA);
    auto q_ptr = c.take<int>(ns + 1); auto q_idx = c.take<int>(nnzQ); auto q_val = c.take<double>(nnzQ);
    auto qf_ptr = c.take<int>(ns + 1); auto qf_idx = c.take<int>(nnzQf); auto qf_val = c.take<double>(nnzQf);
    auto B = c.take<double>((size_t)ns * nu); auto R = c.take<double>((size_t)nu * nu);
    auto xl = c.take<double>(ns); auto xu = c.take<double>(ns);
    auto ul = c.take<double>(nu); auto uu = c.take<double>(nu);
    auto qd = c.take<double>(ns); auto qfd = c.take<double>(ns);
    auto G64 = c.take<double>(G); auto G32 = c.take<float>(G); auto G32lo = c.take<float>(G);
    auto G16 = c.take<__nv_bfloat16>(G);
    auto Gt = c.take<float>(G); auto Gtlo = c.take<float>(G);
    auto H64 = c.take<double>((size_t)n * n); auto H32 = c.take<float>((size_t)n * n);
    auto xbar = c.take<double>(ns); auto y = c.take<double>(SX); auto h = c.take<double>(n);
    auto u = c.take<double>(n); auto x = c.take<double>(SX);
    auto s1 = c.take<double>(SX); auto z1 = c.take<double>(SX);
    auto s2 = c.take<double>(SX); auto z2 = c.take<double>(SX);
    auto s3 = c.take<double>(n); auto z3 = c.take<double>(n);
    auto s4 = c.take<double>(n); auto z4 = c.take<double>(n);
    auto sigx = c.take<double>(SX); auto sigu = c.take<double>(n);
    auto sgu = c.take<double>((size_t)SX + n); auto sgl = c.take<double>((size_t)SX + n);
    auto rsu = c.take<double>((size_t)SX + n); auto rsl = c.take<double>((size_t)SX + n);
    auto rpu = c.take<double>((size_t)SX + n); auto rpl = c.take<double>((size_t)SX + n);
    auto rcu = c.take<double>((size_t)SX + n); auto rcl = c.take<double>((size_t)SX + n);
    auto sigx32 = c.take<float>((size_t)I.N * I.ldg);
    auto wz = c.take<double>(SX); auto wx = c.take<double>(SX);
    auto wzu = c.take<double>(n); auto wxu = c.take<double>(n);
    auto gz = c.take<double>(n); auto gw = c.take<double>(n);
    auto rd = c.take<double>(n); auto b = c.take<double>(n); auto du = c.take<double>(n);
    auto du_aff = c.take<double>(n);
    auto ds1 = c.take<double>(SX); auto dz1 = c.take<double>(SX);
    auto ds2 = c.take<double>(SX); auto dz2 = c.take<double>(SX);
    auto ds3 = c.take<double>(n); auto dz3 = c.take<double>(n);
    auto ds4 = c.take<double>(n); auto dz4 = c.take<double>(n);
    auto M64 = c.take<double>((size_t)n * n); auto M32 = c.take<float>((size_t)n * n);
    auto Xinv32 = c.take<float>((size_t)n * n); auto Tinv32 = c.take<float>((size_t)n * n);
    auto XinvT32 = c.take<float>((size_t)n * n);
    auto rho = c.take<double>(n); auto dcorr = c.take<double>(n); auto mv = c.take<double>(n);
    auto ldiag = c.take<double>(2 * 32 * 32);
    auto pflags = c.take<int>(2 + 32 * 32);   // dataflow Cholesky: epoch, count, flag per row block
    auto mvcnt = c.take<int>((size_t)((ns + 63) / 64) * ((I.N + 15) / 16));   // Gamma v tiles (64 states x 16 stages)
    auto ftasks = c.take<int>(64);
    auto ffw = c.take<float>(4 * (size_t)I.SX);
    auto ffv = c.take<float>(2 * (size_t)n);
    auto pp = c.take<double>(n); auto qq = c.take<double>(n); auto dxs = c.take<double>(SX);
    auto tmpx = c.take<double>(SX);
    auto gpart = c.take<double>(gamma_tmv_part_doubles(ns, n, I.N));
    auto r32 = c.take<float>(n);
    auto Xlo32 = c.take<float>((size_t)n * n); auto XloT32 = c.take<float>((size_t)n * n);
    auto r32lo = c.take<float>(n);
    size_t ws_cc = (size_t)syrk_cc_tiles(n) * cc_splits * 64 * 64 * sizeof(double);
    size_t ws_tc = (size_t)syrk_tc_plan_partials(I.ns, I.nu, I.N) * 128 * 128 * sizeof(float);
    auto tc_plan = c.take<int>(2 * (size_t)syrk_tc_tiles(n) + 2);
    size_t ws = std::max(ws_cc, ws_tc);
    auto syrk_ws = c.take<unsigned char>(ws);
    auto part = c.take<double>((size_t)kParts * kMaxParts);
    auto bar = c.take<unsigned>(6);
    auto sc = c.take<Scal>(1);
    auto trace = c.take<double>((size_t)(max_iter + 1) * kTraceW);
    if (kAssign) {
        I.a_ptr = a_ptr; I.a_idx = a_idx; I.a_val = a_val;
        I.q_ptr = q_ptr; I.q_idx = q_idx; I.q_val = q_val;
        I.qf_ptr = qf_ptr; I.qf_idx = qf_idx; I.qf_val = qf_val;
        I.B = B; I.R = R; I.xl = xl; I.xu = xu; I.ul = ul; I.uu = uu; I.qd = qd; I.qfd = qfd;
        I.G64 = G64; I.G32 = G32; I.G32lo = G32lo; I.G16 = G16; I.Gt = Gt; I.Gtlo = Gtlo; I.H64 = H64; I.H32 = H32;
        I.xbar = xbar; I.y = y; I.h = h; I.u = u; I.x = x;
        I.s1 = s1; I.z1 = z1; I.s2 = s2; I.z2 = z2; I.s3 = s3; I.z3 = z3; I.s4 = s4; I.z4 = z4;
        I.sigx = sigx; I.sigu = sigu; I.sigx32 = sigx32; I.sgu = sgu; I.sgl = sgl;
        I.rsu = rsu; I.rsl = rsl; I.rpu = rpu; I.rpl = rpl; I.rcu = rcu; I.rcl = rcl;
        I.wz = wz; I.wx = wx; I.wzu = wzu; I.wxu = wxu; I.gz = gz; I.gw = gw;
        I.rd = rd; I.b = b; I.du = du; I.du_aff = du_aff;
        I.ds1 = ds1; I.dz1 = dz1; I.ds2 = ds2; I.dz2 = dz2;
        I.ds3 = ds3; I.dz3 = dz3; I.ds4 = ds4; I.dz4 = dz4;
        I.M64 = M64; I.M32 = M32; I.Xinv32 = Xinv32; I.Tinv32 = Tinv32; I.XinvT32 = XinvT32; I.rho = rho; I.dcorr = dcorr; I.mv = mv; I.tmpx = tmpx;
        I.ldiag = ldiag;
        I.pflags = pflags; I.mvcnt = mvcnt;
        I.ftasks = ftasks;
        I.ffw = ffw;
        I.ffv = ffv;
        I.at_ptr = at_ptr; I.at_idx = at_idx; I.at_val = at_val;
        I.bc_ptr = bc_ptr; I.bc_idx = bc_idx; I.bc_val = bc_val;
        I.at_pack = at_pack; I.bc_ff = bc_ff; I.sig_ff = sig_ff;
        I.pp = pp; I.qq = qq; I.dxs = dxs;
        I.gpart = gpart; I.r32 = r32; I.syrk_ws = syrk_ws; I.syrk_ws_bytes = ws;
        I.Xlo32 = Xlo32; I.XloT32 = XloT32; I.r32lo = r32lo;
        I.part = part; I.bar = bar; I.sc = sc; I.trace = trace; I.tc_plan = tc_plan;
    }
    return c.off;
}

// A batch view over one or more contexts.
struct Batch {
    std::vector<lqmpc_ctx*> ctxs;
    Inst* d_insts = nullptr;        // device array
    bool own = false;
    int count = 0, max_ns = 0, max_N = 0, max_n = 0, max_sx = 0, max_total = 0;
    int cc_splits = 1, tc_splits = 1;
    cudaStream_t st = nullptr;
    const void* d_maps = nullptr;   // tensor maps: 3 per instance (BF16, TF32, TF32 low part), instance order
    bool ff = false;                // products with Gamma in float-float (mixed solves) or FP64
    GraphCache* gc = nullptr;       // nullptr: launch every kernel directly
    double warm_mu0 = 0.0;          // > 0: warm start from the guess staged in du_aff
    int potrf_variant[2] = {-1, -1};  // [fp64]: -1 rule, 0 cooperative, 1 cluster, 2 dataflow, 3 queued (autotuned)
    const int* d_ftasks = nullptr;  // queued dataflow Cholesky: task list (nullptr: not available)
    int nftasks = 0;
    bool lyap = false;              // FP64 formation by the Horner chains (every instance's A is sparse enough)
    int max_nu = 0;
    cudaStream_t side = nullptr;    // ctxs[0]'s side stream and events (nullptr: no overlap)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool side_pending = false;      // head work on the side stream not joined yet
    // launches of the conjugate-gradient loop graphs' bodies (counted from
    // the passes the device reports, [FP64 preconditioner])
    unsigned seen_pass[2] = {0u, 0u};
    unsigned long long pass_kernels[2] = {0ull, 0ull};
    // while an iteration is captured into one graph: kernels of the loop
    // bodies captured so far (counted by the pass counters instead), and
    // whether a nested part could not be captured
    unsigned long long loop_body_kernels = 0;
    bool capture_failed = false;
};

// ---- autotuned launch shapes, keyed by batch signature (count and the
// largest dimensions); filled by lqmpc_autotune, optionally from a cache file.
struct Tuning {
    int cc_splits = 0;          // CUDA-core SYRK split-K factor (0: setup heuristic)
    int potrf[2] = {-1, -1};    // potrf variant for FP32 (with inverse) and FP64
    int kkt64 = -1;             // FP64 formation: -1 setup choice, 0 SYRK, 1 backward recursion
};
std::mutex g_tune_mu;
std::map<std::string, Tuning> g_tune;

std::string batch_key(const Batch& b) {
    char k[96];
    snprintf(k, sizeof(k), "b%d-n%d-s%d-N%d", b.count, b.max_n, b.max_ns, b.max_N);
    return k;
}

static bool env_is(const char* k, char c) {
    const char* e = getenv(k);
    return e && e[0] == c;
}

// KKT solves launched without a host read after each (LQMPC_UNSEEN=0: off).
static bool unseen_enabled() {
    static int on = -1;
    if (on < 0) on = env_is("LQMPC_UNSEEN", '0') ? 0 : 1;
    return on == 1;
}

// An unseen iteration captured as one graph (LQMPC_WHOLE=0: off).
static bool whole_iteration_enabled() {
    static int on = -1;
    if (on < 0) on = env_is("LQMPC_WHOLE", '0') ? 0 : 1;
    return on == 1;
}

// Off under the per-launch debug modes (they synchronise or record events per
// launch) or with LQMPC_GRAPH=0.
bool graphs_enabled() {
    static int on = -1;
    if (on < 0) {
        on = !(env_is("LQMPC_GRAPH", '0') || env_is("LQMPC_PROFILE", '1') || env_is("LQMPC_CHECK", '1'));
    }
    return on == 1;
}

// Event-record nodes of a captured graph (the timers around the SYRK and the
// factor, and the iteration's KKT timer) made leaves: each predecessor gets an
// edge straight to each successor and the node keeps only its incoming
// edges.  It still records when its predecessors complete, and no launch
// waits for it (an event node in the chain costs ~4 us between kernels).
static void detach_event_nodes(cudaGraph_t g) {
    if (env_is("LQMPC_DETACH", '0')) return;
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(node, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
        size_t nin = 0, nout = 0;
        cudaGraphNodeGetDependencies(node, nullptr, nullptr, &nin);
        cudaGraphNodeGetDependentNodes(node, nullptr, nullptr, &nout);
        if (nout == 0) continue;
        std::vector<cudaGraphNode_t> in(nin), out(nout);
        if (nin) cudaGraphNodeGetDependencies(node, in.data(), nullptr, &nin);
        cudaGraphNodeGetDependentNodes(node, out.data(), nullptr, &nout);
        for (cudaGraphNode_t o : out) {
            for (cudaGraphNode_t d : in) cudaGraphAddDependencies(g, &d, &o, nullptr, 1);
            cudaGraphRemoveDependencies(g, &node, &o, nullptr, 1);
        }
    }
    cudaGetLastError();   // an edge that existed already
}

static bool is_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive;
}

// Run a fixed launch sequence: the first time under stream capture into a
// graph (then replayed), or directly when graphs are off or capture failed.
// Inside a capture already under way (an iteration captured whole) the
// sequence becomes part of that graph.
template <class F>
void seg_run(const Batch& b, int key, F&& body) {
    if (!b.gc || !graphs_enabled() || is_capturing(b.st)) { body(); return; }
    GraphSeg& g = b.gc->segs[2 * key + (b.ff ? 1 : 0)];   // the Gamma products differ with the arithmetic
    if (g.bad) { body(); return; }
    if (!g.exec) {
        const unsigned long long k0 = lqmpc_kernel_launches();
        if (cudaStreamBeginCapture(b.st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            if (getenv("LQMPC_DEBUG")) fprintf(stderr, "lqmpc: stream capture unavailable on this stream\n");
            cudaGetLastError();
            g.bad = true;
            body();
            return;
        }
        body();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b.st, &graph);
        const unsigned long long nk = lqmpc_kernel_launches() - k0;
        note_launches(-(int)nk);          // captured, not run
        if (e == cudaSuccess && graph) detach_event_nodes(graph);
        if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || !g.exec) {
            if (getenv("LQMPC_DEBUG"))
                fprintf(stderr, "lqmpc: graph capture of segment %d failed (%s); launching directly\n", key,
                        cudaGetErrorString(e));
            cudaGetLastError();
            g.exec = nullptr;
            g.bad = true;
            body();
            return;
        }
        g.kernels = nk;
    }
    if (cudaGraphLaunch(g.exec, b.st) == cudaSuccess) note_launches((int)g.kernels);
}

// The conjugate-gradient loop as one graph: the start (`first`, followed by a
// loop-control launch that restarts the pass count) and a while node whose
// body is `pass` (two steps) plus the loop control, which stops when no
// selected instance is still refining or after `cap` passes.  The host reads
// the instance flags once, after the whole loop.  Returns false (nothing
// launched) when graphs are off or the graph could not be built; the caller
// then runs the loop from the host.
template <class F1, class F2>
bool pcg_loop_graph(const Batch& b, int key, int selr, int cap, int slot, F1&& first, F2&& pass) {
    if (!b.gc || !graphs_enabled()) return false;
    GraphSeg& g = b.gc->segs[2 * key + (b.ff ? 1 : 0)];
    if (g.bad) return false;
    if (!g.exec) {
        auto fail = [&](const char* what, cudaError_t e) {
            if (getenv("LQMPC_DEBUG"))
                fprintf(stderr, "lqmpc: conjugate-gradient loop graph: %s (%s); host loop instead\n", what,
                        cudaGetErrorString(e));
            cudaGetLastError();
            g.bad = true;
            return false;
        };
        const unsigned long long k0 = lqmpc_kernel_launches();
        cudaError_t e = cudaStreamBeginCapture(b.st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return fail("capture", e);
        cudaStreamCaptureStatus cs;
        cudaGraph_t graph = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraphConditionalHandle h = 0;
        e = cudaStreamGetCaptureInfo(b.st, &cs, nullptr, &graph, nullptr, nullptr, nullptr);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
            first();
            launch_pcg_more(b.d_insts, b.count, selr, h, cap, 1, slot, b.st);
            e = cudaStreamGetCaptureInfo(b.st, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
        }
        cudaGraphNode_t wnode = nullptr;
        cudaGraph_t body = nullptr;
        if (e == cudaSuccess) {
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &cp);
            if (e == cudaSuccess) {
                body = cp.conditional.phGraph_out[0];
                e = cudaStreamUpdateCaptureDependencies(b.st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            }
        }
        cudaGraph_t done = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b.st, &done);
        if (e == cudaSuccess) e = e2;
        const unsigned long long n_first = lqmpc_kernel_launches() - k0;
        unsigned long long n_pass = 0;
        if (e == cudaSuccess) {   // the loop body, captured into the while node's graph
            const unsigned long long k1 = lqmpc_kernel_launches();
            e = cudaStreamBeginCaptureToGraph(b.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                pass();
                launch_pcg_more(b.d_insts, b.count, selr, h, cap, 0, slot, b.st);
                cudaGraph_t bg = nullptr;
                e = cudaStreamEndCapture(b.st, &bg);
            }
            n_pass = lqmpc_kernel_launches() - k1;
        }
        note_launches(-(int)(lqmpc_kernel_launches() - k0));   // captured, not run
        if (e == cudaSuccess && done) e = cudaGraphInstantiate(&g.exec, done, 0);
        if (done) cudaGraphDestroy(done);
        if (e != cudaSuccess || !g.exec) {
            g.exec = nullptr;
            return fail("build", e);
        }
        g.kernels = n_first;
        g.pass_kernels = n_pass;
    }
    if (cudaGraphLaunch(g.exec, b.st) != cudaSuccess) return false;
    note_launches((int)g.kernels);
    return true;
}

// The conjugate-gradient loop added to a capture under way (an iteration
// captured whole): `first`, the loop-control launch, and a while node whose
// body (`pass` and the loop control) is captured on a stream of its own.
// Returns false if a part could not be captured (the enclosing capture is
// then discarded, see iter_graph_run).
template <class F1, class F2>
bool pcg_loop_inline(Batch& b, int selr, int cap, int slot, F1&& first, F2&& pass) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraphConditionalHandle h = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(b.st, &cs, nullptr, &graph, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return false;
    first();
    launch_pcg_more(b.d_insts, b.count, selr, h, cap, 1, slot, b.st);
    e = cudaStreamGetCaptureInfo(b.st, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return false;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    e = cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &cp);
    if (e != cudaSuccess) return false;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(b.st, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return false;
    cudaStream_t outer = b.st, aux = nullptr;
    if (cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) != cudaSuccess) return false;
    const unsigned long long k1 = lqmpc_kernel_launches();
    e = cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        b.st = aux;
        pass();
        launch_pcg_more(b.d_insts, b.count, selr, h, cap, 0, slot, b.st);
        b.st = outer;
        cudaGraph_t bg = nullptr;
        e = cudaStreamEndCapture(aux, &bg);
    }
    b.st = outer;
    const unsigned long long n_pass = lqmpc_kernel_launches() - k1;
    cudaStreamDestroy(aux);
    if (e != cudaSuccess) return false;
    b.pass_kernels[slot] = n_pass;
    b.loop_body_kernels += n_pass;
    return true;
}

enum SegKey {
    SEG_HEAD = 1, SEG_HEAD_R = 2, SEG_HEAD_SIDE = 3, SEG_HEAD_CHECK = 4, SEG_FORM = 10 /* + precision */,
    SEG_SOLVE64 = 20, SEG_PCG0 = 30, SEG_PCG2 = 31, SEG_PRED_TAIL = 40, SEG_CORR_TAIL = 50,
    SEG_PCG_LOOP = 60 /* + 100 with the FP64 preconditioner */,
    SEG_ITER = 300 /* + precisions present + 32 with the head on the side stream */
};

// Products with Gamma in the arithmetic of the solve: FP64 for the plain
// FP64 path, float-float on the FP32 pipes for the mixed-precision paths.
// (fuse: kFuse* options, float-float path only)
void gmv(const Batch& b, int in, int out, int flags, int fuse = 0) {
    if (b.ff) launch_gamma_mv_ff(b.d_insts, b.count, b.max_ns, b.max_N, b.max_n, in, out, flags, b.st, fuse);
    else launch_gamma_mv(b.d_insts, b.count, b.max_ns, b.max_N, in, out, flags, b.st);
}

void gtmv(const Batch& b, int w0, int w1, int o0, int o1, int scale0, int flags, int fuse = 0) {
    if (b.ff) launch_gamma_tmv_ff(b.d_insts, b.count, b.max_ns, b.max_N, b.max_n, w0, w1, o0, o1, scale0, flags, b.st, fuse);
    else launch_gamma_tmv(b.d_insts, b.count, b.max_ns, b.max_N, b.max_n, w0, w1, o0, o1, scale0, flags, b.st);
}

// The residual head split across streams: r_p and Sigma (k_resid) on the
// solve's stream, then the Gamma' product and r_d / the right-hand side on
// the side stream while the solve's stream forms and factors M; join_head
// waits for the side stream and runs the stop test (which may finish an
// instance: no kernel of the formation may see that change mid-launch).
void head_fork(Batch& b) {
    seg_run(b, SEG_HEAD_R, [&]() {
        launch_resid_check(b.d_insts, b.count, b.max_total, b.max_n, 1, b.st, true, false, 3, b.ff);
    });
    cudaEventRecord(b.ev_fork, b.st);
    cudaStreamWaitEvent(b.side, b.ev_fork, 0);
    Batch bs = b;
    bs.st = b.side;
    seg_run(bs, SEG_HEAD_SIDE, [&]() {
        gtmv(bs, R_WZ, R_WX, R_GZ, R_GW, 0, F_NONE, kFuseInSplit);   // split by k_resid
        launch_resid_check(bs.d_insts, bs.count, bs.max_total, bs.max_n, 1, bs.st, false, true, 1);
    });
    cudaEventRecord(b.ev_join, b.side);
    b.side_pending = true;
}

void join_head(Batch& b) {
    if (!b.side_pending) return;
    // inside a captured iteration the head's event was recorded before the
    // capture: an external wait node
    cudaStreamWaitEvent(b.st, b.ev_join, is_capturing(b.st) ? cudaEventWaitExternal : 0);
    seg_run(b, SEG_HEAD_CHECK, [&]() {
        launch_resid_check(b.d_insts, b.count, b.max_total, b.max_n, 1, b.st, false, true, 2);
    });
    b.side_pending = false;
}

// M v for the conjugate gradients: Gamma v into tmpx (and dxs when
// to_dxs), then mv = Gamma'(Sigma_x tmpx) and the H and Sigma_u terms (mode
// 0: residual of du, 1: q = M p).  On the float-float path the Sigma_x
// scaling and split ride on the Gamma v sum, the Gamma' sum on the matvec,
// and a direction p split by the preconditioner needs no split launch.
void pcg_apply_m(const Batch& b, int in, int mode, int sel, int selr, bool to_dxs, bool in_split) {
    if (b.ff) {
        const int splits = gamma_tmv_ff_splits(b.count, b.max_ns, b.max_N, b.max_n, 1);
        gmv(b, in, R_TMPX, selr, kFuseOutW | (to_dxs ? kFuseOutDxs : 0) | (in_split ? kFuseInSplit : 0));
        gtmv(b, R_TMPX, R_NONE, R_MV, R_NONE, 1, selr, kFuseInSplit | kFuseNoSum);
        launch_pcg_matvec_ff(b.d_insts, b.count, b.max_n, splits, mode, sel, b.st);
    } else {
        gmv(b, in, R_TMPX, selr);
        gtmv(b, R_TMPX, R_NONE, R_MV, R_NONE, 1, selr);
        if (to_dxs) launch_vec_copy(b.d_insts, b.count, b.max_sx, R_TMPX, R_DXS, 0, sel, b.st);
        launch_pcg_matvec(b.d_insts, b.count, b.max_n, mode, sel, b.st);
    }
}

void batch_dims(Batch& b) {
    b.count = (int)b.ctxs.size();
    b.max_ns = b.max_N = b.max_n = b.max_sx = b.max_total = 0;
    b.cc_splits = b.tc_splits = 1 << 30;
    b.lyap = true;
    b.max_nu = 0;
    for (auto* c : b.ctxs) {
        b.lyap = b.lyap && c->lyap;
        b.max_nu = std::max(b.max_nu, c->h.nu);
        b.max_ns = std::max(b.max_ns, c->h.ns);
        b.max_N = std::max(b.max_N, c->h.N);
        b.max_n = std::max(b.max_n, c->h.n);
        b.max_sx = std::max(b.max_sx, c->h.SX);
        b.max_total = std::max(b.max_total, c->h.SX + c->h.n);
        b.cc_splits = std::min(b.cc_splits, c->cc_splits);
        b.tc_splits = b.tc_splits == (1 << 30) ? c->tc_splits : std::max(b.tc_splits, c->tc_splits);
    }
    if (b.count == 1 && potrf_flowq_fits(b.max_n)) {   // the instance's own task list
        b.d_ftasks = b.ctxs[0]->h.ftasks;
        b.nftasks = flowq_task_count(b.max_n);
    }
    b.st = b.ctxs[0]->stream;
    b.side = b.ctxs[0]->side;
    b.ev_fork = b.ctxs[0]->ev_fork;
    b.ev_join = b.ctxs[0]->ev_join;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(batch_key(b));
    if (it != g_tune.end()) {
        if (it->second.cc_splits > 0 && it->second.cc_splits <= b.cc_splits) b.cc_splits = it->second.cc_splits;
        b.potrf_variant[0] = it->second.potrf[0];
        b.potrf_variant[1] = it->second.potrf[1];
        if (it->second.kkt64 == 0) b.lyap = false;
    }
    // LQMPC_POTRF=coop|cluster|flow|queued fixes the FP32 Cholesky variant
    if (const char* e = getenv("LQMPC_POTRF")) {
        static const char* names[] = {"coop", "cluster", "flow", "queued"};
        for (int v = 0; v < 4; ++v)
            if (!strcmp(e, names[v])) b.potrf_variant[0] = v;
    }
}

// Task list of the queued dataflow Cholesky for a batch: the instances by
// decreasing n (the longest chains start first), none if one is too large.
std::vector<int> batch_flow_tasks(const Batch& b) {
    std::vector<int> order(b.count), t;
    if (!potrf_flowq_fits(b.max_n)) return t;
    for (int i = 0; i < b.count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b.ctxs[x]->h.n > b.ctxs[y]->h.n; });
    for (int q : order) {
        const size_t o = t.size();
        t.resize(o + flowq_task_count(b.ctxs[q]->h.n));
        flowq_tasks(q, b.ctxs[q]->h.n, t.data() + o);
    }
    return t;
}

// ---- one KKT solve M du = b (in role R_B) into R_DU, and R_TMPX = Gamma du.
// Returns false if the mixed-precision refinement did not converge for some
// instance (the caller then falls back to FP64).
// SYRK timing: the events of ctxs[0] bracket the SYRK launch itself.
struct SyrkTimer {
    bool tc = false, cc = false, cc64 = false;   // cc64: the timed CUDA-core launch was FP64
    bool tc3 = false;                            // the timed tensor-core launch was split TF32
    bool pf = false;                             // an FP32 factorisation was timed
};

// Form and factor M in precision `prec` for the instances `sel` picks.
void kkt_form(const Batch& b, int prec, SyrkTimer* tm = nullptr, double shift = 0.0, int sel = F_NONE) {
    lqmpc_ctx* c0 = b.ctxs[0];
    // Under capture the records must be external event nodes (not graph-internal
    // dependencies); the external flag is only valid while capturing.
    auto rec = [&](cudaEvent_t e) {
        if (!tm) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(b.st, &cs);
        if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, b.st, cudaEventRecordExternal);
        else cudaEventRecord(e, b.st);
    };
    auto body = [&]() {
        if (prec == LQMPC_FP32X2) {
            // two-level FP32 preconditioner: M in FP64 (unshifted: E is taken
            // against the exact M), its FP32 rounding (shifted on retries)
            // factored, then the factor of I + X1 E X1' and the combined inverse
            rec(c0->evk[2]);
            if (b.lyap) {
                launch_kkt_lyap_ff(b.d_insts, b.count, b.max_ns, b.max_nu, b.max_N, b.max_sx, sel, b.st, 0.0);
            } else {
                launch_syrk_cc(b.d_insts, b.count, b.max_n, b.cc_splits, 1, 0, nullptr, nullptr, sel, b.st);
                launch_syrk_reduce(b.d_insts, b.count, b.max_n, b.cc_splits, 0, 1, 0, 1, sel, nullptr, b.st, 0.0);
            }
            rec(c0->evk[3]);
            launch_x2_round(b.d_insts, b.count, b.max_n, sel, b.st, shift);
            launch_potrf(b.d_insts, b.count, b.max_n, 0, sel, b.st, 1, b.potrf_variant[0], b.d_ftasks, b.nftasks);
            launch_x2_refine(b.d_insts, b.count, b.max_n, sel, b.st);
            launch_potrf(b.d_insts, b.count, b.max_n, 0, sel, b.st, 1, b.potrf_variant[0], b.d_ftasks, b.nftasks);
            launch_x2_combine(b.d_insts, b.count, b.max_n, sel, b.st);
        } else if (prec == LQMPC_FP64 && b.lyap) {
            rec(c0->evk[2]);
            launch_kkt_lyap(b.d_insts, b.count, b.max_ns, b.max_nu, b.max_N, sel, b.st, shift);
            rec(c0->evk[3]);
            launch_potrf(b.d_insts, b.count, b.max_n, 1, sel, b.st, 0, b.potrf_variant[1], b.d_ftasks, b.nftasks);
        } else if (prec == LQMPC_FP64) {
            rec(c0->evk[2]);
            launch_syrk_cc(b.d_insts, b.count, b.max_n, b.cc_splits, 1, 0, nullptr, nullptr, sel, b.st);
            rec(c0->evk[3]);
            launch_syrk_reduce(b.d_insts, b.count, b.max_n, b.cc_splits, 0, 1, 0, 1, sel, nullptr, b.st, shift);
            launch_potrf(b.d_insts, b.count, b.max_n, 1, sel, b.st, 0, b.potrf_variant[1], b.d_ftasks, b.nftasks);
        } else {
            if (prec == LQMPC_FP32 && !b.d_maps) {
                rec(c0->evk[2]);
                launch_syrk_cc(b.d_insts, b.count, b.max_n, b.cc_splits, 0, 0, nullptr, nullptr, sel, b.st);
                rec(c0->evk[3]);
                launch_syrk_reduce(b.d_insts, b.count, b.max_n, b.cc_splits, 1, 0, 0, 1, sel, nullptr, b.st,
                                   shift);
            } else {
                // FP32: split-TF32 products on the tensor cores (FP32-accurate formation)
                const int mode = prec == LQMPC_MIXED_TF32 ? 1 : (prec == LQMPC_FP32 ? 2 : 0);
                rec(c0->evk[0]);
                launch_syrk_tc(b.d_insts, b.count, b.max_n, b.tc_splits, mode, b.d_maps, sel, b.st);
                rec(c0->evk[1]);
                launch_syrk_reduce(b.d_insts, b.count, b.max_n, b.tc_splits, 2, 0, 0, 1, sel, nullptr, b.st,
                                   shift);
            }
            rec(c0->evk[4]);
            launch_potrf(b.d_insts, b.count, b.max_n, 0, sel, b.st, 1, b.potrf_variant[0], b.d_ftasks, b.nftasks);
            rec(c0->evk[5]);
        }
    };
    // the timed and untimed sequences differ (event nodes): separate graphs
    if (shift == 0.0) seg_run(b, SEG_FORM + prec + (tm ? 5 : 0), body);
    else body();
    if (tm) {
        if (prec == LQMPC_FP64 || prec == LQMPC_FP32X2 || (prec == LQMPC_FP32 && !b.d_maps)) {
            tm->cc = true;
            tm->cc64 = prec == LQMPC_FP64 || prec == LQMPC_FP32X2;
        } else {
            tm->tc = true;
            tm->tc3 = prec == LQMPC_FP32;
        }
        if (prec != LQMPC_FP64 && prec != LQMPC_FP32X2) tm->pf = true;
    }
}

// FP64 factor: the direct solve.
void kkt_solve_fp64(const Batch& b, int sel = F_NONE) {
    seg_run(b, SEG_SOLVE64, [&]() {
        launch_chol_solve(b.d_insts, b.count, b.max_n, 1, R_B, R_DU, sel, b.st);
        gmv(b, R_DU, R_DXS, sel);
    });
}

// Host view of the launch predicate (skip_instance) on a Scal copy.
bool host_selected(const Scal& S, int sel) {
    if (!(sel & F_FORCE) && S.done) return false;
    if ((sel & F_SKIP_REFINED) && (S.refine_ok || S.refine_fail)) return false;
    if ((sel & F_PENDING) && !S.kkt_pending) return false;
    const int mask = (sel >> 8) & 31;
    if (mask && !((mask >> S.prec_cur) & 1)) return false;
    return true;
}

// The copy of every instance's Scal to its host mirror, queued (then
// read_scals_end waits for it, so more work can be queued behind it first).
lqmpc_status read_scals_begin(Batch& b) {
    for (auto* c : b.ctxs) CK(cudaMemcpyAsync(c->h_scal, c->h.sc, sizeof(Scal), cudaMemcpyDeviceToHost, b.st));
    CK(cudaEventRecord(b.ctxs[0]->ev_read, b.st));
    return LQMPC_OK;
}

void count_loop_passes(Batch& b);

lqmpc_status read_scals_end(Batch& b) {
    CK(cudaEventSynchronize(b.ctxs[0]->ev_read));
    count_loop_passes(b);
    return LQMPC_OK;
}

lqmpc_status read_scals(Batch& b) {
    for (auto* c : b.ctxs) CK(cudaMemcpyAsync(c->h_scal, c->h.sc, sizeof(Scal), cudaMemcpyDeviceToHost, b.st));
    CK(cudaStreamSynchronize(b.st));
    count_loop_passes(b);
    return LQMPC_OK;
}

// Launches of the loop graphs' bodies since the last read, from the pass
// counters the device keeps.
void count_loop_passes(Batch& b) {
    const Scal& S0 = *b.ctxs[0]->h_scal;
    for (int k = 0; k < 2; ++k) {
        const unsigned now = (unsigned)S0.pcg_pass_total[k];
        note_launches((int)(b.pass_kernels[k] * (now - b.seen_pass[k])));
        b.seen_pass[k] = now;
    }
}

// Mixed-precision solve of M du = b (R_B -> R_DU, R_DXS = Gamma du):
// preconditioned conjugate gradients with the low-precision Cholesky factor
// as preconditioner and FP64 products with M.  The host looks at the instance
// flags every second step and stops launching once every unfinished instance
// has converged or failed; afterwards each h_scal holds the outcome.
lqmpc_status kkt_solve_mixed(Batch& b, int refine_max, bool prec64 = false, int sel = F_NONE,
                             int budget_lo = -1, int budget_mid = -1, bool unseen = false) {
    if (budget_lo < 0) budget_lo = refine_max;
    if (budget_mid < 0) budget_mid = refine_max;
    const int selr = sel | F_SKIP_REFINED;
    // preconditioner P^{-1}: the FP32 explicit inverse of the low-precision
    // factor, or (prec64) the FP64 triangular solves
    // (tail 1 / 2: then the new direction p from z = P^{-1} r, fused into the
    // FP32 preconditioner's last launch)
    auto prec = [&](int in, int out, int flags, int tail = 0) {
        if (prec64) {
            launch_chol_solve(b.d_insts, b.count, b.max_n, 1, in, out, flags, b.st);
            if (tail == 1) launch_pcg_pinit(b.d_insts, b.count, sel, b.st);
            if (tail == 2) launch_pcg_beta(b.d_insts, b.count, sel, b.st);
        } else {
            launch_prec_apply(b.d_insts, b.count, b.max_n, in, out, flags, b.st, tail);
        }
    };
    const int kp = prec64 ? 100 : 0;   // separate graphs for the two preconditioners
    // start: ||b||, du = P^{-1} b, the initial residual r = b - M du (and
    // Gamma du), z = P^{-1} r and the first direction
    const bool split_du = b.ff && !prec64;   // the FP32 preconditioner splits du for the Gamma du
    auto first = [&]() {
        launch_pcg_begin(b.d_insts, b.count, sel, refine_max, budget_lo, budget_mid, b.st);
        prec(R_B, R_DU, sel, split_du ? 3 : 0);
        pcg_apply_m(b, R_DU, 0, sel, selr, true, split_du);
        prec(R_RHO, R_DCORR, selr, 1);
    };
    // one CG step: q = M p, alpha, du/r/dxs update and test; then z = P r and
    // the new direction (harmless after the last step: every kernel is
    // predicated on the instance's refinement flags)
    auto step = [&](bool with_next) {
        pcg_apply_m(b, R_P, 1, sel, selr, false, !prec64);   // p split by the FP32 preconditioner
        launch_pcg_step_update(b.d_insts, b.count, b.max_total, sel, b.st);
        if (!with_next) return;
        prec(R_RHO, R_DCORR, selr, 2);
    };
    // The start and one step, then two steps at a time.  (Most solves of a
    // mixed-precision run take no step or one: with the first step ahead of
    // the loop a one-step solve enters no pass, and a pass's second step
    // idles only for even counts.)  With graphs the whole loop runs on the
    // device (the passes in a while node) and the host reads the flags once
    // at the end; otherwise the host looks at them after the first step and
    // after every second step, and stops launching once every unfinished
    // instance has converged or failed (the last read leaves each h_scal
    // holding the outcome).
    auto first_step = [&]() {
        first();
        step(true);
    };
    const int cap = refine_max / 2;   // 1 + 2 cap >= refine_max steps (the budgets stop them first)
    if (is_capturing(b.st)) {   // part of an iteration captured whole
        if (!pcg_loop_inline(b, selr, cap, prec64 ? 1 : 0, first_step, [&]() { step(true); step(true); }))
            b.capture_failed = true;
        return LQMPC_OK;
    }
    {
        const int key = SEG_PCG_LOOP + kp, slot = prec64 ? 1 : 0;
        if (pcg_loop_graph(b, key, selr, cap, slot, first_step, [&]() { step(true); step(true); })) {
            b.pass_kernels[slot] = b.gc->segs[2 * key + (b.ff ? 1 : 0)].pass_kernels;
            if (unseen) return LQMPC_OK;   // the outcome is read with the iteration's end
            return read_scals(b);
        }
    }
    seg_run(b, SEG_PCG0 + kp, first_step);
    auto pending = [&]() {
        for (auto* c : b.ctxs)
            if (host_selected(*c->h_scal, selr) && !c->h_scal->info) return true;
        return false;
    };
    lqmpc_status st = read_scals(b);
    if (st != LQMPC_OK) return st;
    for (int s = 1; s < refine_max && pending();) {
        if (s + 2 <= refine_max) {
            seg_run(b, SEG_PCG2 + kp, [&]() { step(true); step(true); });
            s += 2;
        } else {
            step(false);
            s += 1;
        }
        st = read_scals(b);
        if (st != LQMPC_OK) return st;
    }
    return LQMPC_OK;
}

constexpr double kWarmSlackFloor = 1e-2;   // warm start: s0 = max(slack, 1e-2)
constexpr double kWarmMu0 = 1e-2;          // default complementarity of a warm start

// Per-solve preparation: y = Phi xbar, h = Gamma' Qbar y, initial point.
void prepare(const Batch& b, const lqmpc_options& o) {
    for (auto* c : b.ctxs) cudaMemsetAsync(c->h.sc, 0, sizeof(Scal), b.st);
    launch_ychain(b.d_insts, b.count, b.st);
    launch_qbar_y(b.d_insts, b.count, b.max_sx, b.st);
    gtmv(b, R_TMPX, R_NONE, R_H, R_NONE, 0, F_FORCE);
    bool cross = false;
    for (auto* c : b.ctxs) cross = cross || c->h.Sx != nullptr;
    if (cross) launch_h_cross(b.d_insts, b.count, b.max_n, b.st);
    const bool warm = b.warm_mu0 > 0.0;
    launch_set_u0(b.d_insts, b.count, b.max_n, b.st, warm ? 1 : 0);
    gmv(b, R_U, R_TMPX, F_FORCE);
    launch_init_point(b.d_insts, b.count, b.max_total, b.max_n, o.tol, o.tau, o.max_iter, o.refine_tol,
                      o.precision, b.st, warm ? b.warm_mu0 : 0.0, kWarmSlackFloor);
}

constexpr int kLowPrecSteps = 12;   // conjugate-gradient steps allowed with a BF16/TF32 factor
// With fallback on, an FP32 factor gets kFp32Steps steps per solve (the
// two-level tier then costs less than iterating on), and an instance whose
// FP32 solves took more than kFp32IterSteps steps in one interior-point
// iteration (predictor and corrector) moves to the two-level tier for the
// next: the step counts only grow as the iterations close in.
constexpr int kFp32Steps = 8;
constexpr int kFp32IterSteps = 8;

int next_precision(int p) {
    if (p == LQMPC_MIXED_BF16 || p == LQMPC_MIXED_TF32) return LQMPC_FP32;
    return p == LQMPC_FP32 ? LQMPC_FP32X2 : LQMPC_FP64;
}

void write_scal(Batch& b, lqmpc_ctx* c) {
    cudaMemcpyAsync(c->h.sc, c->h_scal, sizeof(Scal), cudaMemcpyHostToDevice, b.st);
}

// Only the precision and the fallback count (the rest of the device Scal may
// be newer than the host's copy).
void write_scal_prec(Batch& b, lqmpc_ctx* c) {
    cudaMemcpyAsync(&c->h.sc->prec_cur, &c->h_scal->prec_cur, sizeof(int), cudaMemcpyHostToDevice, b.st);
    cudaMemcpyAsync(&c->h.sc->fallbacks, &c->h_scal->fallbacks, sizeof(int), cudaMemcpyHostToDevice, b.st);
}

// Form and factor M in precision p (FP32, FP32X2 or FP64) for the instances
// `sel` picks, retried with a relative diagonal shift where a pivot fails
// (an FP64 pivot can fail on rounding when Sigma spans more decades than FP64
// resolves); a shifted FP64 factor is only a preconditioner, so its solves
// are refined (polish).  The host reads the instances after each attempt.
lqmpc_status kkt_form_retried(Batch& b, int p, SyrkTimer* tm, int sel, bool& polish) {
    const double shifts32[3] = {0.0, 1e-6, 1e-4}, shifts64[3] = {0.0, 1e-12, 1e-9};
    const double* shifts = p == LQMPC_FP64 ? shifts64 : shifts32;
    for (int a = 0; a < 3; ++a) {
        if (a > 0 && p == LQMPC_FP64) polish = true;
        kkt_form(b, p, tm, shifts[a], sel);
        join_head(b);
        lqmpc_status st = read_scals(b);
        if (st != LQMPC_OK) return st;
        bool fail = false;
        for (auto* c : b.ctxs)
            if (host_selected(*c->h_scal, sel) && c->h_scal->info) fail = true;
        if (!fail || a == 2) break;
        for (auto* c : b.ctxs)
            if (host_selected(*c->h_scal, sel) && c->h_scal->info) {
                c->h_scal->info = 0;
                write_scal(b, c);
            }
    }
    return LQMPC_OK;
}

// Solve M du = b for every unfinished instance, each with its own factor
// precision (Scal::prec_cur).  Rounds: form and factor M for the instances
// that need it (all of them unless `formed`; later only the escalated ones),
// solve -- FP64 factors directly (or, with `polish`, refined by conjugate
// gradients preconditioned by the FP64 factor), lower precisions by
// conjugate gradients preconditioned by the explicit inverse of the factor --
// then settle.  An instance whose refinement does not converge (or whose
// low-precision Cholesky meets a non-positive pivot even after the FP32
// shift retries) moves to the next precision, BF16/TF32 -> FP32 -> FP32X2
// (the two-level FP32 preconditioner) -> FP64, for
// the rest of the solve (fallback on), or finishes with LQMPC_ERR_STALL /
// LQMPC_ERR_NOT_PD.  Relative diagonal shifts of a retried FP32 factor
// change only the preconditioner: the conjugate gradients with FP64 products
// still converge to the exact solution.  The other instances keep their
// precision: one instance's trouble does not move a whole batch to FP64.
lqmpc_status kkt_step(Batch& b, const lqmpc_options& o, bool formed, SyrkTimer* tm, bool& polish,
                      bool unseen = false) {
    launch_kkt_begin(b.d_insts, b.count, b.st);
    for (auto* c : b.ctxs) c->h_scal->kkt_pending = c->h_scal->done ? 0 : 1;   // the same on the host copy
    const int budget_lo = std::min(o.refine_max, kLowPrecSteps);
    const int budget_mid = o.fallback ? std::min(o.refine_max, kFp32Steps) : o.refine_max;
    if (unseen) {
        // One round, read by the host only at the end of the iteration: the
        // same launches as a round that meets no failing pivot and no
        // refinement that fails; a solve that does fail is marked on the
        // device (spec_fail) and its instance's iteration is repeated.
        int present = 0;
        for (auto* c : b.ctxs)
            if (!c->h_scal->done) present |= 1 << c->h_scal->prec_cur;
        // The factors of the last iterations (FP32X2, FP64) meet failing
        // pivots often enough to be read and retried at once.
        if (!formed)
            for (int p = 0; p < 5; ++p) {
                if (!((present >> p) & 1)) continue;
                const int sel = F_PENDING | prec_sel(1 << p);
                if (p == LQMPC_FP32X2 || p == LQMPC_FP64) {
                    lqmpc_status st = kkt_form_retried(b, p, tm, sel, polish);
                    if (st != LQMPC_OK) return st;
                } else {
                    kkt_form(b, p, tm, 0.0, sel);
                }
            }
        join_head(b);
        if (present & 1) {
            const int sel = F_PENDING | prec_sel(1);
            if (!polish) kkt_solve_fp64(b, sel);
            else {
                lqmpc_status st = kkt_solve_mixed(b, o.refine_max, true, sel, -1, -1, true);
                if (st != LQMPC_OK) return st;
            }
        }
        if (present & 0x1E) {
            lqmpc_status st = kkt_solve_mixed(b, o.refine_max, false, F_PENDING | prec_sel(0x1E), budget_lo,
                                              budget_mid, true);
            if (st != LQMPC_OK) return st;
        }
        launch_kkt_settle(b.d_insts, b.count, b.st, 1);
        for (auto* c : b.ctxs) c->h_scal->kkt_pending = 0;
        return LQMPC_OK;
    }
    for (int round = 0; round < 4; ++round) {
        int present = 0;   // precisions among the pending instances
        for (auto* c : b.ctxs) {
            const Scal& S = *c->h_scal;
            if (!S.done && (round == 0 || S.kkt_pending)) present |= 1 << S.prec_cur;
        }
        if (!present) {
            join_head(b);
            return LQMPC_OK;
        }
        if (!formed || round > 0) {
            for (int p = 0; p < 5; ++p) {
                if (!((present >> p) & 1)) continue;
                const int sel = F_PENDING | prec_sel(1 << p);
                if (p != LQMPC_FP32 && p != LQMPC_FP32X2 && p != LQMPC_FP64) {
                    kkt_form(b, p, tm, 0.0, sel);
                    continue;
                }
                lqmpc_status st = kkt_form_retried(b, p, tm, sel, polish);
                if (st != LQMPC_OK) return st;
            }
        }
        join_head(b);
        if (present & 1) {
            const int sel = F_PENDING | prec_sel(1);
            if (!polish) {
                kkt_solve_fp64(b, sel);
            } else {
                // Near a tight stop tolerance Sigma spreads over many decades
                // and the factorisation of the condensed matrix alone no
                // longer resolves the step.
                lqmpc_status st = kkt_solve_mixed(b, o.refine_max, true, sel);
                if (st != LQMPC_OK) return st;
            }
        }
        if (present & 0x1E) {
            lqmpc_status st =
                kkt_solve_mixed(b, o.refine_max, false, F_PENDING | prec_sel(0x1E), budget_lo, budget_mid);
            if (st != LQMPC_OK) return st;
        }
        // settle on the device and, from the host copies the solves just read
        // (or that no solve since has changed), the same decision here
        launch_kkt_settle(b.d_insts, b.count, b.st, 0);
        for (auto* c : b.ctxs) {
            Scal& S = *c->h_scal;
            if (!S.done && S.kkt_pending && !S.info && (S.prec_cur == LQMPC_FP64 || S.refine_ok)) S.kkt_pending = 0;
        }
        for (auto* c : b.ctxs) {
            Scal& S = *c->h_scal;
            if (S.done || !S.kkt_pending) continue;
            if (S.prec_cur == LQMPC_FP64 || !o.fallback) {
                S.done = 1;
                S.status = S.info ? LQMPC_ERR_NOT_PD : LQMPC_ERR_STALL;
                S.kkt_pending = 0;
            } else {
                S.prec_cur = next_precision(S.prec_cur);
                S.info = 0;
                S.fallbacks += 1;
            }
            write_scal(b, c);
        }
    }
    return LQMPC_OK;
}

// An event record that is an external node when the stream is being
// captured (read by the host after the graph ran).
static void rec_event(cudaEvent_t e, cudaStream_t st) {
    if (is_capturing(st)) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

static int timer_bits(const SyrkTimer& t) {
    return (t.tc ? 1 : 0) | (t.cc ? 2 : 0) | (t.cc64 ? 4 : 0) | (t.tc3 ? 8 : 0) | (t.pf ? 16 : 0);
}
static SyrkTimer timer_from_bits(int v) {
    SyrkTimer t;
    t.tc = v & 1; t.cc = v & 2; t.cc64 = v & 4; t.tc3 = v & 8; t.pf = v & 16;
    return t;
}

// An unseen iteration's launches from the predictor's KKT solve to the step
// as one graph, the conjugate-gradient loops as while nodes inside it (the
// boundaries between separately launched graphs cost 3-6 us each, kernels in
// one graph follow each other within 1 us).  Captured the first time for a
// key and replayed after; when a part cannot be captured the iteration runs
// as separate launches and the key is not tried again.
template <class F>
lqmpc_status iter_graph_run(Batch& b, int key, SyrkTimer& tm, F&& body) {
    GraphSeg& g = b.gc->segs[2 * key + (b.ff ? 1 : 0)];
    if (g.bad) return body();
    if (!g.exec) {
        const unsigned long long k0 = lqmpc_kernel_launches();
        const bool side = b.side_pending;
        b.loop_body_kernels = 0;
        b.capture_failed = false;
        if (cudaStreamBeginCapture(b.st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            g.bad = true;
            return body();
        }
        const lqmpc_status s = body();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(b.st, &graph);
        const unsigned long long nk = lqmpc_kernel_launches() - k0;
        note_launches(-(int)nk);   // captured, not run
        if (e == cudaSuccess && (s != LQMPC_OK || b.capture_failed || !graph)) e = cudaErrorUnknown;
        if (e == cudaSuccess) detach_event_nodes(graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || !g.exec) {
            if (getenv("LQMPC_DEBUG"))
                fprintf(stderr, "lqmpc: capture of a whole iteration failed (%s); separate launches\n",
                        cudaGetErrorString(e));
            cudaGetLastError();
            g.exec = nullptr;
            g.bad = true;
            b.side_pending = side;   // the captured join did not run
            tm = SyrkTimer();
            return body();
        }
        g.kernels = nk - b.loop_body_kernels;   // the loop bodies count by their passes
        g.pass_kernels = b.pass_kernels[0];
        g.timer_bits = timer_bits(tm);
    } else {
        tm = timer_from_bits(g.timer_bits);
        b.pass_kernels[0] = g.pass_kernels;
        b.side_pending = false;   // the graph joins the head
        for (auto* c : b.ctxs) c->h_scal->kkt_pending = 0;
    }
    if (cudaGraphLaunch(g.exec, b.st) != cudaSuccess) return LQMPC_ERR_CUDA;
    note_launches((int)g.kernels);
    return LQMPC_OK;
}

lqmpc_status run_ipm(Batch& b, const lqmpc_options& o, double* t_total, double* t_kkt) {
    const int prec = o.precision;
    b.ff = prec != LQMPC_FP64;
    if ((prec == LQMPC_MIXED_BF16 || prec == LQMPC_MIXED_TF32) && !b.d_maps) return LQMPC_ERR_UNSUPPORTED;
    lqmpc_ctx* c0 = b.ctxs[0];
    c0->t_tc = c0->t_cc = c0->t_cc64 = c0->t_tc3 = c0->t_pf = 0.0;
    c0->n_tc = c0->n_cc = c0->n_cc64 = c0->n_tc3 = c0->n_pf = 0;
    cudaEventRecord(c0->ev[0], b.st);
    // whatever an earlier solve left on the side stream (an error return) is
    // done before this one writes
    if (b.side) cudaStreamWaitEvent(b.st, b.ev_join, 0);
    prepare(b, o);
    {
        lqmpc_status st = read_scals(b);   // host view of the initial per-instance state
        if (st != LQMPC_OK) return st;
    }
    double kkt_ms = 0.0;
    // With graphs the host reads the instance state once per iteration and
    // launches the KKT solves unseen (see kkt_step); after an iteration in
    // which some instance's solve failed, that iteration is repeated with the
    // host looking after every solve.  Repeats do not count against max_iter.
    bool unseen = graphs_enabled() && unseen_enabled();
    int repeats = 0;
    // residuals, Sigma, stop test: on the side stream overlapping the
    // formation, unless an FP64 formation is ahead (it is costly even for the
    // instances it then skips: the stop test's outcome goes to the host first)
    auto fp64_ahead_now = [&]() {
        for (auto* c : b.ctxs)
            if (!c->h_scal->done && (c->h_scal->prec_cur == LQMPC_FP64 || c->h_scal->prec_cur == LQMPC_FP32X2))
                return true;
        return false;
    };
    auto queue_head = [&](bool fp64_ahead) {
        if (b.side && !fp64_ahead) {
            head_fork(b);
        } else {
            seg_run(b, SEG_HEAD, [&]() {
                launch_resid_check(b.d_insts, b.count, b.max_total, b.max_n, 1, b.st, true, false, 3, b.ff);
                gtmv(b, R_WZ, R_WX, R_GZ, R_GW, 0, F_NONE, kFuseInSplit);   // split by k_resid
                launch_resid_check(b.d_insts, b.count, b.max_total, b.max_n, 1, b.st, false, true);
            });
        }
    };
    bool head_queued = false;   // this iteration's head went out behind the last iteration's read
    for (int it = 0; it <= o.max_iter + repeats; ++it) {
        SyrkTimer tm;
        const bool fp64_ahead = fp64_ahead_now();
        if (!head_queued) queue_head(fp64_ahead);
        head_queued = false;
        cudaEventRecord(c0->ev[2], b.st);
        {
            if (fp64_ahead) {
                join_head(b);
                lqmpc_status st = read_scals(b);
                if (st != LQMPC_OK) return st;
                bool all_done = true;
                for (auto* c : b.ctxs)
                    if (!c->h_scal->done) all_done = false;
                if (all_done) break;
            }
        }
        // FP64 solves get a refinement step once mu is within 1e3 of the stop
        // tolerance (the mu of the latest host read)
        bool polish = false;
        for (auto* c : b.ctxs)
            if (!c->h_scal->done && it > 0 && c->h_scal->mu < 1e3 * o.tol) polish = true;
        auto iter_body = [&]() -> lqmpc_status {
            // predictor: form and factor M, solve M du_aff = b
            lqmpc_status st = kkt_step(b, o, false, &tm, polish, unseen);
            if (st != LQMPC_OK) return st;
            seg_run(b, SEG_PRED_TAIL, [&]() {
                // affine step (from the solve's du and Gamma du), sigma,
                // corrector right-hand side
                launch_aff(b.d_insts, b.count, b.max_total, b.st);
                launch_corr(b.d_insts, b.count, b.max_total, b.st, b.ff);
                if (b.ff) {
                    gtmv(b, R_WX, R_NONE, R_GW, R_NONE, 0, F_NONE, kFuseRhs | kFuseInSplit);   // split by k_corr
                } else {
                    gtmv(b, R_WX, R_NONE, R_GW, R_NONE, 0, F_NONE);
                    launch_rhs(b.d_insts, b.count, b.max_n, b.st);
                }
            });
            // corrector: same factor
            st = kkt_step(b, o, true, &tm, polish, unseen);
            if (st != LQMPC_OK) return st;
            rec_event(c0->ev[3], b.st);
            seg_run(b, SEG_CORR_TAIL, [&]() { launch_step_update(b.d_insts, b.count, b.max_total, 1, b.st); });
            return LQMPC_OK;
        };
        // Unseen iterations whose factors need no read in between (no
        // two-level or FP64 tier present) run as one graph.
        int present = 0;
        for (auto* c : b.ctxs)
            if (!c->h_scal->done) present |= 1 << c->h_scal->prec_cur;
        const bool whole = unseen && b.gc && present && !(present & ((1 << LQMPC_FP64) | (1 << LQMPC_FP32X2))) &&
                           whole_iteration_enabled();
        lqmpc_status s = whole ? iter_graph_run(b, SEG_ITER + present + (b.side_pending ? 32 : 0), tm, iter_body)
                               : iter_body();
        if (s != LQMPC_OK) return s;
        // The state goes to the host and the next iteration's head is queued
        // behind it before the host waits, so the GPU runs the head while the
        // host looks.  Its variant comes from the state read an iteration
        // earlier (the variants compute the same values); after the head the
        // host writes back only prec_cur and fallbacks, which it does not touch.
        s = read_scals_begin(b);
        if (s != LQMPC_OK) return s;
        queue_head(fp64_ahead_now());
        head_queued = true;
        s = read_scals_end(b);
        if (s != LQMPC_OK) return s;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c0->ev[2], c0->ev[3]) == cudaSuccess) kkt_ms += ms;
        if (tm.tc && cudaEventElapsedTime(&ms, c0->evk[0], c0->evk[1]) == cudaSuccess) {
            c0->t_tc += ms; c0->n_tc++;
            if (tm.tc3) { c0->t_tc3 += ms; c0->n_tc3++; }
        }
        if (tm.pf && cudaEventElapsedTime(&ms, c0->evk[4], c0->evk[5]) == cudaSuccess) { c0->t_pf += ms; c0->n_pf++; }
        if (tm.cc && cudaEventElapsedTime(&ms, c0->evk[2], c0->evk[3]) == cudaSuccess) {
            c0->t_cc += ms; c0->n_cc++;
            if (tm.cc64) { c0->t_cc64 += ms; c0->n_cc64++; }
        }
        bool all_done = true, failed = false;
        for (auto* c : b.ctxs) {
            if (c->h_scal->err) return LQMPC_ERR_TIMEOUT;
            if (!c->h_scal->done) all_done = false;
            if (!c->h_scal->done && c->h_scal->spec_fail) failed = true;
        }
        if (getenv("LQMPC_DEBUG"))
            for (auto* c : b.ctxs) {
                const Scal& S = *c->h_scal;
                fprintf(stderr, "lqmpc it %d%s: iter %d prec %d spec_fail %d info %d refine ok/fail %d/%d iter_steps %d pending %d fallbacks %d mu %.3e\n",
                        it, unseen ? " (unseen)" : "", S.iter, S.prec_cur, S.spec_fail, S.info, S.refine_ok, S.refine_fail,
                        S.refine_iter, S.kkt_pending, S.fallbacks, S.mu);
            }
        if (all_done) break;
        // An instance whose solve failed unseen repeats the iteration (its
        // iterate was left as it was) with the host looking after every
        // solve: the failing round then runs again and the escalation or the
        // shifted retries follow as without the unseen rounds, so the results
        // are the same.
        if (unseen && failed) ++repeats;
        unseen = graphs_enabled() && unseen_enabled() && !failed;
        // an FP32 instance whose solves grew costly moves on to the two-level tier
        for (auto* c : b.ctxs) {
            Scal& S = *c->h_scal;
            if (o.fallback && !S.done && !S.spec_fail && S.prec_cur == LQMPC_FP32 && S.refine_iter > kFp32IterSteps) {
                S.prec_cur = LQMPC_FP32X2;
                S.fallbacks += 1;
                write_scal_prec(b, c);
            }
        }
    }
    join_head(b);
    cudaEventRecord(c0->ev[1], b.st);
    lqmpc_status s = read_scals(b);
    if (s != LQMPC_OK) return s;
    prof_report(prec == LQMPC_FP64 ? "fp64 solve" : "mixed solve");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c0->ev[0], c0->ev[1]);
    *t_total = ms;
    *t_kkt = kkt_ms;
    if (cudaGetLastError() != cudaSuccess) return LQMPC_ERR_CUDA;
    return LQMPC_OK;
}

void fill_stats(lqmpc_ctx* c, lqmpc_stats* st, double t_total, double t_kkt) {
    const Scal& S = *c->h_scal;
    if (!st) return;
    st->iters = S.iter;
    st->refine_steps = S.refine_steps;
    st->fallbacks = S.fallbacks;
    st->status = S.done ? S.status : LQMPC_ERR_MAXITER;
    st->mu = S.mu;
    st->res_primal = S.res_p;
    st->res_dual = S.res_d;
    st->t_total_ms = t_total;
    st->t_kkt_ms = t_kkt;
    st->t_syrk_tc_ms = c->t_tc;
    st->t_syrk_cc_ms = c->t_cc;
    st->syrk_tc_launches = c->n_tc;
    st->syrk_cc_launches = c->n_cc;
    st->t_syrk_fp64_ms = c->t_cc64;
    st->syrk_fp64_launches = c->n_cc64;
    st->t_syrk_tc3_ms = c->t_tc3;
    st->syrk_tc3_launches = c->n_tc3;
    st->t_potrf32_ms = c->t_pf;
    st->potrf32_launches = c->n_pf;
}

lqmpc_status final_status(lqmpc_ctx* c) {
    const Scal& S = *c->h_scal;
    if (!S.done) return LQMPC_ERR_MAXITER;
    return (lqmpc_status)S.status;
}

// The input sequence of the last solve into dst: the solver's variable, or
// with a feedback K the lifted rows u_t = K x_t + v_t of x_{t+1}.
cudaError_t copy_u(const lqmpc_ctx* c, double* dst, cudaMemcpyKind kind, cudaStream_t st) {
    const Inst& I = c->h;
    if (c->u_row < 0) return cudaMemcpyAsync(dst, I.u, sizeof(double) * I.n, kind, st);
    return cudaMemcpy2DAsync(dst, sizeof(double) * I.nu, I.x + c->u_row, sizeof(double) * I.ns,
                             sizeof(double) * I.nu, I.N, kind, st);
}

lqmpc_status solve_common(lqmpc_ctx* ctx, const double* x0, bool x0_dev, double* u, bool u_dev,
                          lqmpc_stats* st, const double* u_init = nullptr, double mu0 = 0.0) {
    if (!ctx || !x0 || !u) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    const Inst& I = ctx->h;
    const int nsp = ctx->ns_plant;   // x0 holds the plant's states; lifted rows start at zero
    if (!x0_dev) {
        if (!all_finite(x0, nsp)) return LQMPC_ERR_ARG;
        CK(cudaMemcpyAsync(I.xbar, x0, sizeof(double) * nsp, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        CK(cudaMemcpyAsync(I.xbar, x0, sizeof(double) * nsp, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (I.ns > nsp) CK(cudaMemsetAsync(I.xbar + nsp, 0, sizeof(double) * (I.ns - nsp), ctx->stream));
    if (u_init) {
        if (ctx->u_row >= 0) return LQMPC_ERR_UNSUPPORTED;   // the guess would be for v, not u
        if (!all_finite(u_init, I.n)) return LQMPC_ERR_ARG;
        CK(cudaMemcpyAsync(I.du_aff, u_init, sizeof(double) * I.n, cudaMemcpyHostToDevice, ctx->stream));
    }
    Batch b;
    b.ctxs = {ctx};
    b.d_insts = ctx->d_inst;
    batch_dims(b);
    b.d_maps = ctx->tc_ok ? ctx->d_maps : nullptr;
    if (!ctx->graphs) ctx->graphs = new (std::nothrow) GraphCache();
    b.gc = ctx->graphs;
    if (u_init) b.warm_mu0 = mu0 > 0.0 ? mu0 : kWarmMu0;
    double tt = 0, tk = 0;
    lqmpc_status s = run_ipm(b, ctx->opts, &tt, &tk);
    if (s != LQMPC_OK) return s;
    CK(copy_u(ctx, u, u_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    fill_stats(ctx, st, tt, tk);
    return final_status(ctx);
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

lqmpc_options lqmpc_default_options(void) {
    lqmpc_options o;
    o.tol = 1e-8;
    o.max_iter = 100;
    o.precision = LQMPC_FP64;
    o.refine_max = 30;
    o.refine_tol = 1e-10;
    o.fallback = 1;
    o.tau = 0.995;
    o.verbose = 0;
    return o;
}

const char* lqmpc_status_str(int s) {
    switch (s) {
        case LQMPC_OK: return "ok";
        case LQMPC_ERR_ARG: return "invalid argument";
        case LQMPC_ERR_CUDA: return "CUDA error";
        case LQMPC_ERR_NOT_PD: return "KKT matrix not positive definite";
        case LQMPC_ERR_MAXITER: return "iteration limit reached";
        case LQMPC_ERR_INFEASIBLE: return "infeasible";
        case LQMPC_ERR_NAN: return "non-finite iterate";
        case LQMPC_ERR_STALL: return "iterative refinement stalled";
        case LQMPC_ERR_TIMEOUT: return "device wait timed out";
        case LQMPC_ERR_UNSUPPORTED: return "unsupported option or size";
        default: return "unknown status";
    }
}

static bool opts_ok(const lqmpc_options& o) {
    return o.tol > 0 && o.max_iter >= 1 && o.max_iter <= 100000 && o.precision >= 0 && o.precision <= 4 &&
           o.refine_max >= 0 && o.refine_max <= 100 && o.refine_tol > 0 && o.tau > 0 && o.tau < 1;
}

static lqmpc_status setup_impl(lqmpc_ctx** out, int ns, int nu, int N, const int* a_ptr, const int* a_idx,
                               const double* a_val, const double* Bh, const int* q_ptr, const int* q_idx,
                               const double* q_val, const int* qf_ptr, const int* qf_idx, const double* qf_val,
                               const double* Rh, const double* xl, const double* xu, const double* ul,
                               const double* uu, const lqmpc_options* opts, void* stream, const double* Sh,
                               const double* wh) {
    if (!out) return LQMPC_ERR_ARG;
    *out = nullptr;
    if (ns < 1 || nu < 1 || N < 1 || (long long)nu * N > 30000 || (long long)ns * N > (1LL << 31) - 1)
        return LQMPC_ERR_ARG;
    if (!Bh || !Rh || !xl || !xu || !ul || !uu) return LQMPC_ERR_ARG;
    if (!csr_ok(ns, a_ptr, a_idx, a_val) || !csr_ok(ns, q_ptr, q_idx, q_val)) return LQMPC_ERR_ARG;
    const bool qf_given = qf_ptr != nullptr;
    if (qf_given && !csr_ok(ns, qf_ptr, qf_idx, qf_val)) return LQMPC_ERR_ARG;
    if (!all_finite(Bh, (size_t)ns * nu) || !all_finite(Rh, (size_t)nu * nu)) return LQMPC_ERR_ARG;
    for (int i = 0; i < ns; ++i)
        if (std::isnan(xl[i]) || std::isnan(xu[i]) || xl[i] > xu[i] || xl[i] == INFINITY || xu[i] == -INFINITY)
            return LQMPC_ERR_ARG;
    for (int j = 0; j < nu; ++j)
        if (std::isnan(ul[j]) || std::isnan(uu[j]) || ul[j] > uu[j] || ul[j] == INFINITY || uu[j] == -INFINITY)
            return LQMPC_ERR_ARG;
    lqmpc_options o = opts ? *opts : lqmpc_default_options();
    if (!opts_ok(o)) return LQMPC_ERR_ARG;
    if (!qf_given) { qf_ptr = q_ptr; qf_idx = q_idx; qf_val = q_val; }

    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) return LQMPC_ERR_CUDA;
    lqmpc_ctx* ctx = new (std::nothrow) lqmpc_ctx();
    if (!ctx) return LQMPC_ERR_CUDA;
    cudaGetDevice(&ctx->device);
    ctx->user_stream = (cudaStream_t)stream;
    ctx->stream = (cudaStream_t)stream;
    if (!stream) {
        // Own blocking stream: it stays ordered with the legacy default stream
        // (where the caller's work goes) and, unlike it, can be captured into
        // CUDA graphs.
        if (cudaStreamCreate(&ctx->stream) != cudaSuccess) {
            delete ctx;
            return LQMPC_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    ctx->opts = o;
    Inst& I = ctx->h;
    memset(&I, 0, sizeof(I));
    I.ns = ns; I.nu = nu; I.N = N; I.n = nu * N; I.SX = ns * N;
    I.ldg = (int)align_up(ns, 64);
    std::vector<double> qd, qfd;
    bool qdiag = csr_diag(ns, q_ptr, q_idx, q_val, qd) && csr_diag(ns, qf_ptr, qf_idx, qf_val, qfd);
    I.q_diag = qdiag ? 1 : 0;
    const int nnzA = a_ptr[ns], nnzQ = q_ptr[ns], nnzQf = qf_ptr[ns];
    ctx->cc_splits = syrk_cc_splits(ns, nu, N);
    ctx->tc_splits = syrk_tc_plan_partials(ns, nu, N);
    // A' in CSR (the columns of A) and the nonzeros of B per column, for the
    // backward-recursion formation of the FP64 KKT matrix
    std::vector<int> at_ptr(ns + 1, 0), at_idx(nnzA), bc_ptr(nu + 1, 0), bc_idx;
    std::vector<double> at_val(nnzA), bc_val;
    for (int k = 0; k < nnzA; ++k) at_ptr[a_idx[k] + 1]++;
    for (int i = 0; i < ns; ++i) at_ptr[i + 1] += at_ptr[i];
    {
        std::vector<int> fill(at_ptr.begin(), at_ptr.end() - 1);
        for (int r = 0; r < ns; ++r)
            for (int k = a_ptr[r]; k < a_ptr[r + 1]; ++k) {
                const int q = fill[a_idx[k]]++;
                at_idx[q] = r;
                at_val[q] = a_val[k];
            }
    }
    for (int col = 0; col < nu; ++col) {
        for (int i = 0; i < ns; ++i)
            if (Bh[(size_t)col * ns + i] != 0.0) {
                bc_idx.push_back(i);
                bc_val.push_back(Bh[(size_t)col * ns + i]);
            }
        bc_ptr[col + 1] = (int)bc_idx.size();
    }
    const int nnzB = (int)bc_idx.size();
    // the Horner chains when they need fewer FP64 operations than the SYRK, or
    // when both are small (a batch forms all its FP64 instances one way, so one
    // small instance should not move the others to the SYRK); LQMPC_KKT64=
    // syrk|lyap overrides
    {
        const double cs = kkt_cost_syrk(ns, nu, N), cl = kkt_cost_lyap(ns, nu, N, nnzA, nnzB);
        ctx->lyap = cl < cs || cl < 4e6;
        if (const char* e = getenv("LQMPC_KKT64")) {
            if (!strcmp(e, "syrk")) ctx->lyap = false;
            if (!strcmp(e, "lyap")) ctx->lyap = true;
        }
    }
    size_t bytes = layout<false>(I, nullptr, nnzA, nnzQ, nnzQf, o.max_iter, ctx->cc_splits, ctx->tc_splits, nnzB,
                                 ctx->lyap);
    auto fail = [&](lqmpc_status s) {
        lqmpc_free(ctx);
        return s;
    };
    if (cudaMalloc(&ctx->arena, bytes) != cudaSuccess) return fail(LQMPC_ERR_CUDA);
    ctx->arena_bytes = bytes;
    if (cudaMemsetAsync(ctx->arena, 0, bytes, ctx->stream) != cudaSuccess) return fail(LQMPC_ERR_CUDA);
    layout<true>(I, ctx->arena, nnzA, nnzQ, nnzQf, o.max_iter, ctx->cc_splits, ctx->tc_splits, nnzB, ctx->lyap);
    if (cudaMallocHost(&ctx->h_scal, sizeof(Scal)) != cudaSuccess) return fail(LQMPC_ERR_CUDA);
    memset(ctx->h_scal, 0, sizeof(Scal));
    for (int e = 0; e < 6; ++e)
        if ((e < 4 && cudaEventCreate(&ctx->ev[e]) != cudaSuccess) || cudaEventCreate(&ctx->evk[e]) != cudaSuccess)
            return fail(LQMPC_ERR_CUDA);
    ctx->events = true;
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_read, cudaEventDisableTiming) != cudaSuccess)
        return fail(LQMPC_ERR_CUDA);
    cudaStream_t st = ctx->stream;
    auto up = [&](const void* dst, const void* src, size_t n) {
        return cudaMemcpyAsync((void*)dst, src, n, cudaMemcpyHostToDevice, st) == cudaSuccess;
    };
    bool ok = up(I.a_ptr, a_ptr, sizeof(int) * (ns + 1)) && up(I.a_idx, a_idx, sizeof(int) * nnzA) &&
              up(I.a_val, a_val, sizeof(double) * nnzA) && up(I.q_ptr, q_ptr, sizeof(int) * (ns + 1)) &&
              up(I.q_idx, q_idx, sizeof(int) * nnzQ) && up(I.q_val, q_val, sizeof(double) * nnzQ) &&
              up(I.qf_ptr, qf_ptr, sizeof(int) * (ns + 1)) && up(I.qf_idx, qf_idx, sizeof(int) * nnzQf) &&
              up(I.qf_val, qf_val, sizeof(double) * nnzQf) && up(I.B, Bh, sizeof(double) * ns * nu) &&
              up(I.R, Rh, sizeof(double) * nu * nu) && up(I.xl, xl, sizeof(double) * ns) &&
              up(I.xu, xu, sizeof(double) * ns) && up(I.ul, ul, sizeof(double) * nu) &&
              up(I.uu, uu, sizeof(double) * nu);
    if (qdiag) ok = ok && up(I.qd, qd.data(), sizeof(double) * ns) && up(I.qfd, qfd.data(), sizeof(double) * ns);
    ok = ok && up(I.at_ptr, at_ptr.data(), sizeof(int) * (ns + 1)) && up(I.at_idx, at_idx.data(), sizeof(int) * nnzA) &&
         up(I.at_val, at_val.data(), sizeof(double) * nnzA) && up(I.bc_ptr, bc_ptr.data(), sizeof(int) * (nu + 1)) &&
         up(I.bc_idx, bc_idx.data(), sizeof(int) * nnzB) && up(I.bc_val, bc_val.data(), sizeof(double) * nnzB);
    {   // float-float splits (hi plane, then lo plane) for the float-float Horner chains
        auto split = [](const std::vector<double>& v) {
            std::vector<float> f(2 * v.size());
            for (size_t k = 0; k < v.size(); ++k) {
                f[k] = (float)v[k];
                f[v.size() + k] = (float)(v[k] - (double)f[k]);
            }
            return f;
        };
        const std::vector<float> af = split(at_val), bf = split(bc_val);
        std::vector<int> pack(4 * (size_t)nnzA, 0);
        for (int k = 0; k < nnzA; ++k) {
            pack[4 * (size_t)k] = at_idx[k];
            memcpy(&pack[4 * (size_t)k + 1], &af[k], sizeof(float));
            memcpy(&pack[4 * (size_t)k + 2], &af[nnzA + k], sizeof(float));
        }
        ok = ok && up(I.at_pack, pack.data(), sizeof(int) * pack.size()) &&
             up(I.bc_ff, bf.data(), sizeof(float) * bf.size());
    }
    {
        std::vector<int> plan = syrk_tc_make_plan(ns, nu, N);
        ok = ok && up(I.tc_plan, plan.data(), sizeof(int) * plan.size());
    }
    if (potrf_flowq_fits(I.n)) {
        std::vector<int> ft(flowq_task_count(I.n));
        flowq_tasks(0, I.n, ft.data());
        ok = ok && up(I.ftasks, ft.data(), sizeof(int) * ft.size());
    }
    if (!ok) return fail(LQMPC_ERR_CUDA);
    if (Sh || wh) {   // general data: S (ns x nu) and w (N x ns)
        const size_t sn = Sh ? (size_t)ns * nu : 0, wn = wh ? (size_t)N * ns : 0;
        if (cudaMalloc(&ctx->gen_dev, sizeof(double) * (sn + wn)) != cudaSuccess) return fail(LQMPC_ERR_CUDA);
        if (Sh && !up(ctx->gen_dev, Sh, sizeof(double) * sn)) return fail(LQMPC_ERR_CUDA);
        if (wh && !up(ctx->gen_dev + sn, wh, sizeof(double) * wn)) return fail(LQMPC_ERR_CUDA);
        I.Sx = Sh ? ctx->gen_dev : nullptr;
        I.wd = wh ? ctx->gen_dev + sn : nullptr;
    }
    if (cudaMalloc(&ctx->d_inst, sizeof(Inst)) != cudaSuccess) return fail(LQMPC_ERR_CUDA);
    if (!up(ctx->d_inst, &I, sizeof(Inst))) return fail(LQMPC_ERR_CUDA);
    // the solve's Scal starts "not done" for the setup-time launches
    cudaMemsetAsync(I.sc, 0, sizeof(Scal), st);

    // one-time state elimination and H (FP64)
    launch_gstack(ctx->d_inst, I, st);
    if (qdiag) {
        launch_syrk_cc(ctx->d_inst, 1, I.n, ctx->cc_splits, 1, 1, nullptr, nullptr, F_FORCE, st);
    } else {
        double *gq = nullptr, *gqf = nullptr;
        size_t gb = sizeof(double) * (size_t)I.ldg * I.n;
        if (cudaMalloc(&gq, gb) != cudaSuccess || cudaMalloc(&gqf, gb) != cudaSuccess) {
            cudaFree(gq);
            return fail(LQMPC_ERR_CUDA);
        }
        cudaMemsetAsync(gq, 0, gb, st);
        cudaMemsetAsync(gqf, 0, gb, st);
        launch_q_times_g(ctx->d_inst, I, 0, gq, st);
        launch_q_times_g(ctx->d_inst, I, 1, gqf, st);
        launch_syrk_cc(ctx->d_inst, 1, I.n, ctx->cc_splits, 1, 2, gq, gqf, F_FORCE, st);
        cudaStreamSynchronize(st);
        cudaFree(gq);
        cudaFree(gqf);
    }
    launch_syrk_reduce(ctx->d_inst, 1, I.n, ctx->cc_splits, 0, 1, 1, 0, F_FORCE, I.H64, st);
    if (Sh) launch_hess_cross(ctx->d_inst, I.n, st);   // + the stage cross term x_t' S u_t
    launch_h_to_f32(ctx->d_inst, I.n, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(LQMPC_ERR_CUDA);
    // tensor maps for the tcgen05 SYRK (BF16 and TF32 views of the G-stack)
    {
        alignas(64) unsigned char maps[3 * 128];
        bool m0 = syrk_tc_make_maps(I, 0, maps);
        bool m1 = syrk_tc_make_maps(I, 1, maps + 128);
        bool m2 = syrk_tc_make_maps(I, 2, maps + 256);
        if (m0 && m1 && m2) {
            if (cudaMalloc(&ctx->d_maps, sizeof(maps)) != cudaSuccess) return fail(LQMPC_ERR_CUDA);
            if (cudaMemcpy(ctx->d_maps, maps, sizeof(maps), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(LQMPC_ERR_CUDA);
            ctx->tc_ok = 1;
        }
    }
    ctx->ns_plant = ns;   // lqmpc_setup_general sets the caller's dimension after this
    *out = ctx;
    return LQMPC_OK;
}

lqmpc_status lqmpc_setup(lqmpc_ctx** out, int ns, int nu, int N, const int* a_ptr, const int* a_idx,
                         const double* a_val, const double* Bh, const int* q_ptr, const int* q_idx,
                         const double* q_val, const int* qf_ptr, const int* qf_idx, const double* qf_val,
                         const double* Rh, const double* xl, const double* xu, const double* ul,
                         const double* uu, const lqmpc_options* opts, void* stream) {
    return setup_impl(out, ns, nu, N, a_ptr, a_idx, a_val, Bh, q_ptr, q_idx, q_val, qf_ptr, qf_idx, qf_val, Rh, xl,
                      xu, ul, uu, opts, stream, nullptr, nullptr);
}

// General data of Eq. 1 by a lifting to the box-constrained form the solver
// runs: the nc general rows of stage t become extra states of x_{t+1},
// c_{t+1} = E x_t + F u_t (rows [E 0] of the lifted A, F of the lifted B, no
// cost, bounds [gl, gu]); a feedback K (u_t = K x_t + v_t, Section II)
// becomes A + B K, Q + S K + K' S' + K' R K, cross term S + K' R, general
// rows E + F K and nu more lifted rows c = K x_t + v_t = u_t carrying the
// input bounds (v itself is free); the cross term and the disturbance go to
// the device as they are.
lqmpc_status lqmpc_setup_general(lqmpc_ctx** out, int ns, int nu, int N, const int* a_ptr, const int* a_idx,
                                 const double* a_val, const double* Bh, const int* q_ptr, const int* q_idx,
                                 const double* q_val, const int* qf_ptr, const int* qf_idx, const double* qf_val,
                                 const double* Rh, const double* xl, const double* xu, const double* ul,
                                 const double* uu, const lqmpc_general* g, const lqmpc_options* opts,
                                 void* stream) {
    if (!out) return LQMPC_ERR_ARG;
    *out = nullptr;
    if (!g) return setup_impl(out, ns, nu, N, a_ptr, a_idx, a_val, Bh, q_ptr, q_idx, q_val, qf_ptr, qf_idx, qf_val,
                              Rh, xl, xu, ul, uu, opts, stream, nullptr, nullptr);
    if (ns < 1 || nu < 1 || N < 1 || g->nc < 0 || g->nc > (1 << 20)) return LQMPC_ERR_ARG;
    if (!Bh || !Rh || !xl || !xu || !ul || !uu) return LQMPC_ERR_ARG;
    if (!csr_ok(ns, a_ptr, a_idx, a_val) || !csr_ok(ns, q_ptr, q_idx, q_val)) return LQMPC_ERR_ARG;
    if (qf_ptr && !csr_ok(ns, qf_ptr, qf_idx, qf_val)) return LQMPC_ERR_ARG;
    const int nc = g->nc;
    if (nc > 0 && (!g->E || !g->F || !g->gl || !g->gu)) return LQMPC_ERR_ARG;
    if ((g->S && !all_finite(g->S, (size_t)ns * nu)) || (g->w && !all_finite(g->w, (size_t)N * ns)) ||
        (g->K && !all_finite(g->K, (size_t)nu * ns)) || !all_finite(Bh, (size_t)ns * nu) ||
        !all_finite(Rh, (size_t)nu * nu))
        return LQMPC_ERR_ARG;
    if (nc > 0 && (!all_finite(g->E, (size_t)nc * ns) || !all_finite(g->F, (size_t)nc * nu))) return LQMPC_ERR_ARG;
    for (int r = 0; r < nc; ++r)
        if (std::isnan(g->gl[r]) || std::isnan(g->gu[r]) || g->gl[r] > g->gu[r] || g->gl[r] == INFINITY ||
            g->gu[r] == -INFINITY)
            return LQMPC_ERR_ARG;
    const double* K = g->K;
    const int ncu = K ? nu : 0;           // lifted input rows
    const int nca = nc + ncu;             // all lifted rows
    const int nsa = ns + nca;
    if (!qf_ptr) { qf_ptr = q_ptr; qf_idx = q_idx; qf_val = q_val; }
    // dense copies where K mixes the data
    auto dense_of = [&](const int* p, const int* ix, const double* v) {
        std::vector<double> d((size_t)ns * ns, 0.0);
        for (int r = 0; r < ns; ++r)
            for (int k = p[r]; k < p[r + 1]; ++k) d[r + (size_t)ix[k] * ns] += v[k];
        return d;
    };
    // rows of the lifted A, B, Q, Qf as (row, col, value) lists
    std::vector<std::vector<std::pair<int, double>>> Ar(nsa), Qr(nsa), Qfr(nsa);
    std::vector<double> Ba((size_t)nsa * nu, 0.0), Sa;
    bool has_S = g->S != nullptr;
    if (!K) {
        for (int r = 0; r < ns; ++r) {
            for (int k = a_ptr[r]; k < a_ptr[r + 1]; ++k) Ar[r].push_back({a_idx[k], a_val[k]});
            for (int k = q_ptr[r]; k < q_ptr[r + 1]; ++k) Qr[r].push_back({q_idx[k], q_val[k]});
        }
        if (has_S) Sa.assign(g->S, g->S + (size_t)ns * nu);
    } else {
        std::vector<double> Ad = dense_of(a_ptr, a_idx, a_val), Qd = dense_of(q_ptr, q_idx, q_val);
        for (int i = 0; i < ns; ++i)           // A + B K
            for (int j = 0; j < ns; ++j) {
                double v = Ad[i + (size_t)j * ns];
                for (int a = 0; a < nu; ++a) v += Bh[i + (size_t)a * ns] * K[a + (size_t)j * nu];
                Ad[i + (size_t)j * ns] = v;
            }
        std::vector<double> RK((size_t)nu * ns, 0.0);   // R K
        for (int a = 0; a < nu; ++a)
            for (int j = 0; j < ns; ++j) {
                double v = 0.0;
                for (int b = 0; b < nu; ++b) v += Rh[a + (size_t)b * nu] * K[b + (size_t)j * nu];
                RK[a + (size_t)j * nu] = v;
            }
        Sa.assign((size_t)ns * nu, 0.0);       // S + K' R
        for (int i = 0; i < ns; ++i)
            for (int a = 0; a < nu; ++a) {
                double v = g->S ? g->S[i + (size_t)a * ns] : 0.0;
                for (int b = 0; b < nu; ++b) v += K[b + (size_t)i * nu] * Rh[b + (size_t)a * nu];
                Sa[i + (size_t)a * ns] = v;
            }
        has_S = true;
        for (int i = 0; i < ns; ++i)           // Q + S K + K' S' + K' R K
            for (int j = 0; j < ns; ++j) {
                double v = Qd[i + (size_t)j * ns];
                for (int a = 0; a < nu; ++a) {
                    const double sk = g->S ? g->S[i + (size_t)a * ns] * K[a + (size_t)j * nu] +
                                                 g->S[j + (size_t)a * ns] * K[a + (size_t)i * nu]
                                           : 0.0;
                    v += sk + K[a + (size_t)i * nu] * RK[a + (size_t)j * nu];
                }
                Qd[i + (size_t)j * ns] = v;
            }
        for (int i = 0; i < ns; ++i)
            for (int j = 0; j < ns; ++j) {
                if (Ad[i + (size_t)j * ns] != 0.0) Ar[i].push_back({j, Ad[i + (size_t)j * ns]});
                if (Qd[i + (size_t)j * ns] != 0.0) Qr[i].push_back({j, Qd[i + (size_t)j * ns]});
            }
    }
    for (int r = 0; r < ns; ++r)
        for (int k = qf_ptr[r]; k < qf_ptr[r + 1]; ++k) Qfr[r].push_back({qf_idx[k], qf_val[k]});
    for (int i = 0; i < ns; ++i)
        for (int a = 0; a < nu; ++a) Ba[i + (size_t)a * nsa] = Bh[i + (size_t)a * ns];
    std::vector<double> xla(nsa), xua(nsa), ula(nu), uua(nu);
    for (int i = 0; i < ns; ++i) { xla[i] = xl[i]; xua[i] = xu[i]; }
    for (int r = 0; r < nc; ++r) {             // general rows: E + F K, F
        const int row = ns + r;
        for (int j = 0; j < ns; ++j) {
            double v = g->E[r + (size_t)j * nc];
            if (K)
                for (int a = 0; a < nu; ++a) v += g->F[r + (size_t)a * nc] * K[a + (size_t)j * nu];
            if (v != 0.0) Ar[row].push_back({j, v});
        }
        for (int a = 0; a < nu; ++a) Ba[row + (size_t)a * nsa] = g->F[r + (size_t)a * nc];
        xla[row] = g->gl[r];
        xua[row] = g->gu[r];
    }
    for (int a = 0; a < ncu; ++a) {            // u_t = K x_t + v_t, bounds [ul, uu]
        const int row = ns + nc + a;
        for (int j = 0; j < ns; ++j)
            if (K[a + (size_t)j * nu] != 0.0) Ar[row].push_back({j, K[a + (size_t)j * nu]});
        Ba[row + (size_t)a * nsa] = 1.0;
        xla[row] = ul[a];
        xua[row] = uu[a];
    }
    for (int a = 0; a < nu; ++a) {
        ula[a] = K ? -INFINITY : ul[a];
        uua[a] = K ? INFINITY : uu[a];
    }
    auto to_csr = [&](const std::vector<std::vector<std::pair<int, double>>>& rows, std::vector<int>& p,
                      std::vector<int>& ix, std::vector<double>& v) {
        p.assign(nsa + 1, 0);
        for (int r = 0; r < nsa; ++r) {
            for (auto& e : rows[r]) { ix.push_back(e.first); v.push_back(e.second); }
            p[r + 1] = (int)ix.size();
        }
    };
    std::vector<int> ap, ai, qp, qi, fp, fi;
    std::vector<double> av, qv, fv;
    to_csr(Ar, ap, ai, av);
    to_csr(Qr, qp, qi, qv);
    to_csr(Qfr, fp, fi, fv);
    std::vector<double> Sl, wl;
    if (has_S) {
        Sl.assign((size_t)nsa * nu, 0.0);
        for (int i = 0; i < ns; ++i)
            for (int a = 0; a < nu; ++a) Sl[i + (size_t)a * nsa] = Sa[i + (size_t)a * ns];
    }
    if (g->w) {
        wl.assign((size_t)N * nsa, 0.0);
        for (int t = 0; t < N; ++t)
            for (int i = 0; i < ns; ++i) wl[(size_t)t * nsa + i] = g->w[(size_t)t * ns + i];
    }
    lqmpc_status s = setup_impl(out, nsa, nu, N, ap.data(), ai.data(), av.data(), Ba.data(), qp.data(), qi.data(),
                                qv.data(), fp.data(), fi.data(), fv.data(), Rh, xla.data(), xua.data(), ula.data(),
                                uua.data(), opts, stream, has_S ? Sl.data() : nullptr, g->w ? wl.data() : nullptr);
    if (s == LQMPC_OK && K) (*out)->u_row = ns + nc;
    if (s == LQMPC_OK) (*out)->ns_plant = ns;
    return s;
}

lqmpc_status lqmpc_set_options(lqmpc_ctx* ctx, const lqmpc_options* opts) {
    if (!ctx || !opts || !opts_ok(*opts)) return LQMPC_ERR_ARG;
    if (opts->max_iter > ctx->opts.max_iter) return LQMPC_ERR_ARG;  // trace buffer sized at setup
    ctx->opts = *opts;
    return LQMPC_OK;
}

lqmpc_status lqmpc_solve(lqmpc_ctx* ctx, const double* x0, double* u_out, lqmpc_stats* stats) {
    return solve_common(ctx, x0, false, u_out, false, stats);
}

lqmpc_status lqmpc_solve_device(lqmpc_ctx* ctx, const double* x0_device, double* u_device,
                                lqmpc_stats* stats) {
    return solve_common(ctx, x0_device, true, u_device, true, stats);
}

lqmpc_status lqmpc_solve_warm(lqmpc_ctx* ctx, const double* x0, const double* u_init, double mu0, double* u_out,
                              lqmpc_stats* stats) {
    if (!u_init || std::isnan(mu0)) return LQMPC_ERR_ARG;
    return solve_common(ctx, x0, false, u_out, false, stats, u_init, mu0);
}

static lqmpc_status solve_batch_impl(lqmpc_ctx* const* ctxs, int count, const double* const* x0s,
                                     const double* const* u_inits, double mu0, double* const* u_outs,
                                     lqmpc_stats* stats) {
    if (!ctxs || count < 1 || !x0s || !u_outs) return LQMPC_ERR_ARG;
    if (u_inits) {
        if (std::isnan(mu0)) return LQMPC_ERR_ARG;
        for (int i = 0; i < count; ++i)
            if (!u_inits[i] || (ctxs[i] && !all_finite(u_inits[i], ctxs[i]->h.n))) return LQMPC_ERR_ARG;
        for (int i = 0; i < count; ++i)
            if (ctxs[i] && ctxs[i]->u_row >= 0) return LQMPC_ERR_UNSUPPORTED;
    }
    for (int i = 0; i < count; ++i)
        if (!ctxs[i] || !x0s[i] || !u_outs[i] || ctxs[i]->user_stream != ctxs[0]->user_stream ||
            ctxs[i]->device != ctxs[0]->device)
            return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctxs[0]->device));
    for (int i = 1; i < count; ++i)      // contexts with streams of their own: nothing may be in flight
        if (ctxs[i]->stream != ctxs[0]->stream) CK(cudaStreamSynchronize(ctxs[i]->stream));
    Batch b;
    b.ctxs.assign(ctxs, ctxs + count);
    batch_dims(b);
    lqmpc_options o = ctxs[0]->opts;
    for (int i = 0; i < count; ++i) {
        if (!all_finite(x0s[i], ctxs[i]->ns_plant)) return LQMPC_ERR_ARG;
        if (ctxs[i]->opts.max_iter < o.max_iter) o.max_iter = ctxs[i]->opts.max_iter;
    }
    // tensor maps for the tensor-core formations (BF16, TF32 and the split-TF32
    // FP32 tier, which falls back to the CUDA-core SYRK without them)
    bool tc = o.precision == LQMPC_MIXED_BF16 || o.precision == LQMPC_MIXED_TF32 || o.precision == LQMPC_FP32;
    for (int i = 0; i < count && tc; ++i)
        if (!ctxs[i]->tc_ok) tc = false;
    if ((o.precision == LQMPC_MIXED_BF16 || o.precision == LQMPC_MIXED_TF32) && !tc) o.precision = LQMPC_FP32;
    std::vector<Inst> hosts(count);
    for (int i = 0; i < count; ++i) hosts[i] = ctxs[i]->h;
    Inst* d = nullptr;
    void* maps = nullptr;
    const std::vector<int> ftasks = count > 1 ? batch_flow_tasks(b) : std::vector<int>();
    CK(cudaMalloc(&d, sizeof(Inst) * count + sizeof(int) * ftasks.size()));
    if (!ftasks.empty()) {
        b.d_ftasks = reinterpret_cast<const int*>(d + count);
        b.nftasks = (int)ftasks.size();
    }
    if (tc && count > 1 && cudaMalloc(&maps, 384 * (size_t)count) != cudaSuccess) {
        cudaFree(d);
        return LQMPC_ERR_CUDA;
    }
    b.d_insts = d;
    lqmpc_status s = LQMPC_OK;
    if (tc) {
        // every instance's two tensor maps, in instance order (the kernel indexes them by blockIdx.y)
        if (count == 1) b.d_maps = ctxs[0]->d_maps;
        else {
            for (int i = 0; i < count && s == LQMPC_OK; ++i)
                if (cudaMemcpyAsync((char*)maps + 384 * (size_t)i, ctxs[i]->d_maps, 384, cudaMemcpyDeviceToDevice,
                                    b.st) != cudaSuccess)
                    s = LQMPC_ERR_CUDA;
            b.d_maps = maps;
        }
    }
    if (cudaMemcpyAsync(d, hosts.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, b.st) != cudaSuccess)
        s = LQMPC_ERR_CUDA;
    if (!ftasks.empty() && cudaMemcpyAsync(d + count, ftasks.data(), sizeof(int) * ftasks.size(),
                                           cudaMemcpyHostToDevice, b.st) != cudaSuccess)
        s = LQMPC_ERR_CUDA;
    for (int i = 0; i < count && s == LQMPC_OK; ++i) {
        const int nsp = ctxs[i]->ns_plant, nsl = ctxs[i]->h.ns;   // plant states given, lifted rows zero
        if (cudaMemcpyAsync(ctxs[i]->h.xbar, x0s[i], sizeof(double) * nsp, cudaMemcpyHostToDevice, b.st) !=
                cudaSuccess ||
            (nsl > nsp &&
             cudaMemsetAsync(ctxs[i]->h.xbar + nsp, 0, sizeof(double) * (nsl - nsp), b.st) != cudaSuccess))
            s = LQMPC_ERR_CUDA;
    }
    if (u_inits) {      // warm start: every instance's guess where prepare() reads it
        for (int i = 0; i < count && s == LQMPC_OK; ++i)
            if (cudaMemcpyAsync(ctxs[i]->h.du_aff, u_inits[i], sizeof(double) * ctxs[i]->h.n,
                                cudaMemcpyHostToDevice, b.st) != cudaSuccess)
                s = LQMPC_ERR_CUDA;
        b.warm_mu0 = mu0 > 0.0 ? mu0 : kWarmMu0;
    }
    double tt = 0, tk = 0;
    {
        GraphCache gc;      // graphs of this call's descriptor array
        b.gc = &gc;
        if (s == LQMPC_OK) s = run_ipm(b, o, &tt, &tk);
        b.gc = nullptr;
    }
    if (s == LQMPC_OK) {
        for (int i = 0; i < count; ++i)
            if (copy_u(ctxs[i], u_outs[i], cudaMemcpyDeviceToHost, b.st) != cudaSuccess)
                s = LQMPC_ERR_CUDA;
        if (cudaStreamSynchronize(b.st) != cudaSuccess) s = LQMPC_ERR_CUDA;
    }
    cudaFree(d);
    cudaFree(maps);
    if (s != LQMPC_OK) return s;
    lqmpc_status first = LQMPC_OK;
    for (int i = 0; i < count; ++i) {
        if (stats) fill_stats(ctxs[i], &stats[i], tt, tk);
        lqmpc_status si = final_status(ctxs[i]);
        if (si != LQMPC_OK && first == LQMPC_OK) first = si;
    }
    return first;
}

lqmpc_status lqmpc_solve_batch(lqmpc_ctx* const* ctxs, int count, const double* const* x0s,
                               double* const* u_outs, lqmpc_stats* stats) {
    return solve_batch_impl(ctxs, count, x0s, nullptr, 0.0, u_outs, stats);
}

lqmpc_status lqmpc_solve_batch_warm(lqmpc_ctx* const* ctxs, int count, const double* const* x0s,
                                    const double* const* u_inits, double mu0, double* const* u_outs,
                                    lqmpc_stats* stats) {
    if (!u_inits) return LQMPC_ERR_ARG;
    return solve_batch_impl(ctxs, count, x0s, u_inits, mu0, u_outs, stats);
}

lqmpc_status lqmpc_autotune(lqmpc_ctx* const* ctxs, int count, const char* cache_path) {
    if (!ctxs || count < 1) return LQMPC_ERR_ARG;
    for (int i = 0; i < count; ++i)
        if (!ctxs[i] || ctxs[i]->user_stream != ctxs[0]->user_stream || ctxs[i]->device != ctxs[0]->device)
            return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctxs[0]->device));
    for (int i = 1; i < count; ++i)
        if (ctxs[i]->stream != ctxs[0]->stream) CK(cudaStreamSynchronize(ctxs[i]->stream));
    Batch b;
    b.ctxs.assign(ctxs, ctxs + count);
    batch_dims(b);
    const std::string key = batch_key(b);
    // cached decisions
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char k[128];
            int cc, p32, p64, k64;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            while (fscanf(f, "%127s %d %d %d %d", k, &cc, &p32, &p64, &k64) == 5) {
                Tuning t;
                t.cc_splits = cc; t.potrf[0] = p32; t.potrf[1] = p64; t.kkt64 = k64;
                g_tune[k] = t;
            }
            fclose(f);
            if (g_tune.count(key)) return LQMPC_OK;
        }
    }
    const int max_splits = b.cc_splits;   // the smallest workspace of the batch
    b.potrf_variant[0] = b.potrf_variant[1] = -1;
    std::vector<Inst> hosts(count);
    for (int i = 0; i < count; ++i) hosts[i] = ctxs[i]->h;
    Inst* d = nullptr;
    const std::vector<int> ftasks = count > 1 ? batch_flow_tasks(b) : std::vector<int>();
    CK(cudaMalloc(&d, sizeof(Inst) * count + sizeof(int) * ftasks.size()));
    b.d_insts = d;
    if (!ftasks.empty()) {
        b.d_ftasks = reinterpret_cast<const int*>(d + count);
        b.nftasks = (int)ftasks.size();
    }
    lqmpc_status s = LQMPC_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((!ftasks.empty() && cudaMemcpyAsync(d + count, ftasks.data(), sizeof(int) * ftasks.size(),
                                            cudaMemcpyHostToDevice, b.st) != cudaSuccess) ||
        cudaMemcpyAsync(d, hosts.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, b.st) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        s = LQMPC_ERR_CUDA;
    Tuning t;
    if (s == LQMPC_OK) {
        // a representative Sigma: the cold initial point (x0 = 0) and its residuals
        for (auto* c : b.ctxs) cudaMemsetAsync(c->h.xbar, 0, sizeof(double) * c->h.ns, b.st);
        lqmpc_options o = ctxs[0]->opts;
        prepare(b, o);
        launch_resid_check(b.d_insts, b.count, b.max_total, b.max_n, 0, b.st, true, false);
        // best of three timed launches of fn; `pre` (untimed) restores the input
        auto timed = [&](const std::function<void()>& pre, const std::function<void()>& fn) {
            float best = 1e30f;
            for (int r = 0; r < 3; ++r) {
                if (pre) pre();
                cudaEventRecord(e0, b.st);
                fn();
                cudaEventRecord(e1, b.st);
                float ms = 0.f;
                if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    best = std::min(best, ms);
            }
            return best;
        };
        // 1. split-K factor of the CUDA-core SYRK (FP32 formation + reduce)
        float best = 1e30f;
        std::vector<int> cand;
        for (int c = 1; c <= max_splits; c *= 2) cand.push_back(c);
        if (cand.empty() || cand.back() != max_splits) cand.push_back(max_splits);
        for (int c : cand) {
            float ms = timed(nullptr, [&]() {
                launch_syrk_cc(b.d_insts, b.count, b.max_n, c, 0, 0, nullptr, nullptr, F_NONE, b.st);
                launch_syrk_reduce(b.d_insts, b.count, b.max_n, c, 1, 0, 0, 1, F_NONE, nullptr, b.st);
            });
            if (ms < best) { best = ms; t.cc_splits = c; }
        }
        b.cc_splits = t.cc_splits;
        // 2. Cholesky variant: cooperative over all SMs, one 8-CTA cluster per
        //    instance (in a batch with larger instances: clusters for those
        //    that fit, the queued or cooperative kernel for the rest), or (FP32
        //    with the inverse) the dataflow kernel of one instance and the
        //    queued dataflow kernel
        const bool flowq = b.d_ftasks && potrf_flowq_fits(b.max_n);
        if (potrf_cluster_fits(b.max_n) || potrf_flow_fits(b.count, b.max_n) || flowq || b.count > 1) {
            for (int fp64 = 0; fp64 < 2; ++fp64) {
                float bv = 1e30f;
                for (int v = 0; v < 4; ++v) {
                    if (v == 1 && !potrf_cluster_fits(b.max_n) && b.count == 1) continue;
                    if (v == 2 && (fp64 || !potrf_flow_fits(b.count, b.max_n))) continue;
                    if (v == 3 && (fp64 || !flowq)) continue;
                    auto form = [&]() {
                        const int prec = fp64 ? LQMPC_FP64 : LQMPC_FP32;
                        launch_syrk_cc(b.d_insts, b.count, b.max_n, b.cc_splits, fp64, 0, nullptr, nullptr, F_NONE,
                                       b.st);
                        launch_syrk_reduce(b.d_insts, b.count, b.max_n, b.cc_splits, fp64 ? 0 : 1, fp64, 0, 1,
                                           F_NONE, nullptr, b.st);
                        (void)prec;
                    };
                    float ms = timed(form, [&]() {
                        launch_potrf(b.d_insts, b.count, b.max_n, fp64, F_NONE, b.st, fp64 ? 0 : 1, v, b.d_ftasks,
                                     b.nftasks);
                    });
                    if (ms < bv) { bv = ms; t.potrf[fp64] = v; }
                }
            }
        } else {
            t.potrf[0] = t.potrf[1] = 0;
        }
        // 3. FP64 formation: SYRK or backward recursion (where every instance has its buffers)
        if (b.lyap) {
            const float ts = timed(nullptr, [&]() {
                launch_syrk_cc(b.d_insts, b.count, b.max_n, b.cc_splits, 1, 0, nullptr, nullptr, F_NONE, b.st);
                launch_syrk_reduce(b.d_insts, b.count, b.max_n, b.cc_splits, 0, 1, 0, 1, F_NONE, nullptr, b.st);
            });
            const float tl = timed(nullptr, [&]() {
                launch_kkt_lyap(b.d_insts, b.count, b.max_ns, b.max_nu, b.max_N, F_NONE, b.st);
            });
            t.kkt64 = tl < ts ? 1 : 0;
        }
        if (cudaStreamSynchronize(b.st) != cudaSuccess || cudaGetLastError() != cudaSuccess) s = LQMPC_ERR_CUDA;
        // the autotune launches left the instances mid-setup: mark them not started
        for (auto* c : b.ctxs) cudaMemsetAsync(c->h.sc, 0, sizeof(Scal), b.st);
        cudaStreamSynchronize(b.st);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (s != LQMPC_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = t;
    }
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d %d %d\n", key.c_str(), t.cc_splits, t.potrf[0], t.potrf[1], t.kkt64);
            fclose(f);
        }
    }
    return LQMPC_OK;
}

unsigned long long lqmpc_kernel_launches(void) { return g_launches.load(); }

void lqmpc_free(lqmpc_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    delete ctx->graphs;
    ctx->graphs = nullptr;
    if (ctx->events)
        for (int e = 0; e < 6; ++e) {
            if (e < 4) cudaEventDestroy(ctx->ev[e]);
            cudaEventDestroy(ctx->evk[e]);
        }
    cudaFree(ctx->arena);
    cudaFree(ctx->gen_dev);
    cudaFree(ctx->d_inst);
    cudaFree(ctx->d_maps);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_read) cudaEventDestroy(ctx->ev_read);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// ---------------------------------------------------------------------------
// Stage-level entry points
// ---------------------------------------------------------------------------

lqmpc_status lqmpc_get_gstack(lqmpc_ctx* ctx, double* G) {
    if (!ctx || !G) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    const Inst& I = ctx->h;
    std::vector<double> raw((size_t)I.ldg * I.n);
    CK(cudaMemcpy(raw.data(), I.G64, sizeof(double) * raw.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < I.N; ++k)
        for (int c = 0; c < I.nu; ++c)
            memcpy(G + ((size_t)k * I.nu + c) * I.ns, raw.data() + (size_t)I.ldg * ((I.N - 1 - k) * I.nu + c),
                   sizeof(double) * I.ns);
    return LQMPC_OK;
}

lqmpc_status lqmpc_get_hessian(lqmpc_ctx* ctx, double* H) {
    if (!ctx || !H) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpy(H, ctx->h.H64, sizeof(double) * ctx->h.n * ctx->h.n, cudaMemcpyDeviceToHost));
    return LQMPC_OK;
}

static lqmpc_status reset_scal(lqmpc_ctx* ctx) {
    Scal s;
    memset(&s, 0, sizeof(s));
    s.refine_tol = ctx->opts.refine_tol;
    s.tol = ctx->opts.tol;
    s.tau = ctx->opts.tau;
    s.max_iter = ctx->opts.max_iter;
    CK(cudaMemcpyAsync(ctx->h.sc, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LQMPC_OK;
}

lqmpc_status lqmpc_gamma_mv(lqmpc_ctx* ctx, const double* v, double* out) {
    if (!ctx || !v || !out) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    const Inst& I = ctx->h;
    lqmpc_status s = reset_scal(ctx);
    if (s) return s;
    CK(cudaMemcpyAsync(I.du, v, sizeof(double) * I.n, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->opts.precision != LQMPC_FP64)
        launch_gamma_mv_ff(ctx->d_inst, 1, I.ns, I.N, I.n, R_DU, R_TMPX, F_FORCE, ctx->stream);
    else
        launch_gamma_mv(ctx->d_inst, 1, I.ns, I.N, R_DU, R_TMPX, F_FORCE, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, I.tmpx, sizeof(double) * I.SX, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LQMPC_OK;
}

lqmpc_status lqmpc_gamma_tmv(lqmpc_ctx* ctx, const double* w, double* out) {
    if (!ctx || !w || !out) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    const Inst& I = ctx->h;
    lqmpc_status s = reset_scal(ctx);
    if (s) return s;
    CK(cudaMemcpyAsync(I.tmpx, w, sizeof(double) * I.SX, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->opts.precision != LQMPC_FP64)
        launch_gamma_tmv_ff(ctx->d_inst, 1, I.ns, I.N, I.n, R_TMPX, R_NONE, R_MV, R_NONE, 0, F_FORCE, ctx->stream);
    else
        launch_gamma_tmv(ctx->d_inst, 1, I.ns, I.N, I.n, R_TMPX, R_NONE, R_MV, R_NONE, 0, F_FORCE, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, I.mv, sizeof(double) * I.n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LQMPC_OK;
}

static lqmpc_status upload_sigma(lqmpc_ctx* ctx, const double* sigx, const double* sigu) {
    const Inst& I = ctx->h;
    if (!all_finite(sigx, I.SX) || !all_finite(sigu, I.n)) return LQMPC_ERR_ARG;
    for (int k = 0; k < I.SX; ++k)
        if (sigx[k] < 0) return LQMPC_ERR_ARG;
    for (int k = 0; k < I.n; ++k)
        if (sigu[k] < 0) return LQMPC_ERR_ARG;
    std::vector<float> s32((size_t)I.N * I.ldg, 0.0f);
    for (int r = 0; r < I.N; ++r)
        for (int i = 0; i < I.ns; ++i) s32[(size_t)r * I.ldg + i] = (float)sigx[(size_t)r * I.ns + i];
    CK(cudaMemcpyAsync(I.sigx, sigx, sizeof(double) * I.SX, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(I.sigx32, s32.data(), sizeof(float) * s32.size(), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(I.sigu, sigu, sizeof(double) * I.n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LQMPC_OK;
}

static lqmpc_status download_matrix(lqmpc_ctx* ctx, bool fp64, double* out, bool lower_only) {
    const Inst& I = ctx->h;
    size_t nn = (size_t)I.n * I.n;
    if (fp64) {
        CK(cudaMemcpy(out, I.M64, sizeof(double) * nn, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> t(nn);
        CK(cudaMemcpy(t.data(), I.M32, sizeof(float) * nn, cudaMemcpyDeviceToHost));
        for (size_t q = 0; q < nn; ++q) out[q] = t[q];
        // the FP32 formations may write the lower triangle only: mirror it
        if (!lower_only)
            for (int k = 0; k < I.n; ++k)
                for (int j = 0; j < k; ++j) out[j + (size_t)I.n * k] = out[k + (size_t)I.n * j];
    }
    if (lower_only)
        for (int k = 0; k < I.n; ++k)
            for (int j = 0; j < k; ++j) out[j + (size_t)I.n * k] = 0.0;
    return LQMPC_OK;
}

lqmpc_status lqmpc_form_kkt(lqmpc_ctx* ctx, const double* sigx, const double* sigu, int precision,
                            double* M) {
    if (!ctx || !sigx || !sigu || !M || precision < 0 || precision > 4) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    if ((precision == LQMPC_MIXED_BF16 || precision == LQMPC_MIXED_TF32) && !ctx->tc_ok)
        return LQMPC_ERR_UNSUPPORTED;
    if (precision == LQMPC_FP32X2 && !ctx->lyap) return LQMPC_ERR_UNSUPPORTED;
    lqmpc_status s = upload_sigma(ctx, sigx, sigu);
    if (s) return s;
    s = reset_scal(ctx);
    if (s) return s;
    Batch b;
    b.ctxs = {ctx};
    b.d_insts = ctx->d_inst;
    batch_dims(b);
    b.d_maps = ctx->d_maps;
    const Inst& I = ctx->h;
    if (precision == LQMPC_FP64) {
        launch_syrk_cc(b.d_insts, 1, I.n, b.cc_splits, 1, 0, nullptr, nullptr, F_NONE, b.st);
        launch_syrk_reduce(b.d_insts, 1, I.n, b.cc_splits, 0, 1, 0, 1, F_NONE, nullptr, b.st);
    } else if (precision == LQMPC_FP32X2) {
        launch_kkt_lyap_ff(b.d_insts, 1, I.ns, I.nu, I.N, I.SX, F_NONE, b.st, 0.0);
    } else if (precision == LQMPC_FP32 && !ctx->tc_ok) {
        launch_syrk_cc(b.d_insts, 1, I.n, b.cc_splits, 0, 0, nullptr, nullptr, F_NONE, b.st);
        launch_syrk_reduce(b.d_insts, 1, I.n, b.cc_splits, 1, 0, 0, 1, F_NONE, nullptr, b.st);
    } else {
        // the solves' tensor-core formation: BF16, TF32, or split TF32 for the FP32 tier
        const int mode = precision == LQMPC_MIXED_TF32 ? 1 : (precision == LQMPC_FP32 ? 2 : 0);
        launch_syrk_tc(b.d_insts, 1, I.n, b.tc_splits, mode, b.d_maps, F_NONE, b.st);
        launch_syrk_reduce(b.d_insts, 1, I.n, b.tc_splits, 2, 0, 0, 1, F_NONE, nullptr, b.st);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(b.st));
    return download_matrix(ctx, precision == LQMPC_FP64 || precision == LQMPC_FP32X2, M, false);
}

lqmpc_status lqmpc_form_kkt_noalloc(lqmpc_ctx* ctx, const double* sigx, const double* sigu, double* M) {
    if (!ctx || !sigx || !sigu || !M) return LQMPC_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(sigx) | reinterpret_cast<uintptr_t>(sigu) | reinterpret_cast<uintptr_t>(M)) & 7)
        return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    const Inst& I = ctx->h;
    const int r = launch_form_kkt_noalloc(I.G64, I.ldg, I.H64, sigx, sigu, M, I.ns, I.nu, I.N, ctx->stream);
    if (r == 1) {
        if (ctx->opts.verbose)
            fprintf(stderr, "lqmpc_form_kkt_noalloc: n = %d exceeds the fixed scratch (n <= %d)\n", I.n,
                    noalloc_max_n());
        return LQMPC_ERR_UNSUPPORTED;
    }
    return r == 0 ? LQMPC_OK : LQMPC_ERR_CUDA;
}

lqmpc_status lqmpc_kkt_solve(lqmpc_ctx* ctx, const double* sigx, const double* sigu, int precision,
                             const double* rhs, double* x, double* L, int* refine_steps) {
    if (!ctx || !sigx || !sigu || !rhs || !x || precision < 0 || precision > 4) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    if ((precision == LQMPC_MIXED_BF16 || precision == LQMPC_MIXED_TF32) && !ctx->tc_ok)
        return LQMPC_ERR_UNSUPPORTED;
    const Inst& I = ctx->h;
    if (!all_finite(rhs, I.n)) return LQMPC_ERR_ARG;
    lqmpc_status s = upload_sigma(ctx, sigx, sigu);
    if (s) return s;
    s = reset_scal(ctx);
    if (s) return s;
    Batch b;
    b.ctxs = {ctx};
    b.d_insts = ctx->d_inst;
    batch_dims(b);
    b.d_maps = ctx->d_maps;
    CK(cudaMemcpyAsync(I.b, rhs, sizeof(double) * I.n, cudaMemcpyHostToDevice, b.st));
    b.ff = precision != LQMPC_FP64;
    kkt_form(b, precision);
    if (precision == LQMPC_FP64) kkt_solve_fp64(b);
    else {
        lqmpc_status rs = kkt_solve_mixed(b, ctx->opts.refine_max);
        if (rs != LQMPC_OK) return rs;
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_scal, I.sc, sizeof(Scal), cudaMemcpyDeviceToHost, b.st));
    CK(cudaStreamSynchronize(b.st));
    CK(cudaMemcpy(x, I.du, sizeof(double) * I.n, cudaMemcpyDeviceToHost));
    if (L) {
        s = download_matrix(ctx, precision == LQMPC_FP64, L, true);
        if (s) return s;
    }
    if (refine_steps) *refine_steps = ctx->h_scal->refine_steps;
    if (ctx->h_scal->info) return LQMPC_ERR_NOT_PD;
    if (precision != LQMPC_FP64 && !ctx->h_scal->refine_ok) return LQMPC_ERR_STALL;
    return LQMPC_OK;
}

lqmpc_status lqmpc_get_trace(lqmpc_ctx* ctx, double* trace, int max_rows, int* rows) {
    if (!ctx || !trace || !rows || max_rows < 0) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    Scal S;
    CK(cudaMemcpy(&S, ctx->h.sc, sizeof(S), cudaMemcpyDeviceToHost));
    int r = std::min(S.iter + 1, ctx->opts.max_iter + 1);
    r = std::min(r, max_rows);
    if (r > 0) CK(cudaMemcpy(trace, ctx->h.trace, sizeof(double) * kTraceW * r, cudaMemcpyDeviceToHost));
    *rows = r;
    return LQMPC_OK;
}

lqmpc_status lqmpc_get_duals(lqmpc_ctx* ctx, double* z) {
    if (!ctx || !z) return LQMPC_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    const Inst& I = ctx->h;
    CK(cudaMemcpy(z, I.z1, sizeof(double) * I.SX, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(z + I.SX, I.z2, sizeof(double) * I.SX, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(z + 2 * (size_t)I.SX, I.z3, sizeof(double) * I.n, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(z + 2 * (size_t)I.SX + I.n, I.z4, sizeof(double) * I.n, cudaMemcpyDeviceToHost));
    return LQMPC_OK;
}

}  // extern "C"
