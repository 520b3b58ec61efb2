// Host side of libtacta: plans, the CTA / TA / minimum-norm drivers and the C ABI.
//
// The drivers enqueue the per-iteration kernels of kernels.cu on the caller's
// stream. All decisions of the algorithms (stop tests, pivot test, rho growth,
// the auxiliary solve) are taken on the device by finisher code, so the host
// never waits inside an iteration: it enqueues blocks of iterations (replayed
// as a captured CUDA graph by default) and reads a 4-byte stop flag once per
// block, one block behind, so the GPU always has queued work.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"
#include "hankel.cuh"
#include "dia_plan.cuh"

namespace tacta {

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* get_error() { return g_err.c_str(); }

// ------------------------------------------------------------------ per-device one-time setup
static std::mutex g_done_lock;
static std::set<std::pair<const void*, int>> g_done;

bool done_on_device(const void* key) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> guard(g_done_lock);
    return g_done.count({key, dev}) != 0;
}

void mark_done_on_device(const void* key) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> guard(g_done_lock);
    g_done.insert({key, dev});
}

#define CUDA_TRY(expr)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                  \
            return e_ == cudaErrorMemoryAllocation ? TACTA_ERR_OOM : TACTA_ERR_CUDA;        \
        }                                                                                   \
    } while (0)

// ------------------------------------------------------------------ kernels local to the driver
__global__ void ctl_set_trip(Ctl* c, double rho, int max_iter) {
    c->rho = rho;
    c->max_iter = max_iter;
    c->status = 0;
    c->k = 0;
    c->pivot = 0;
    c->need_true = 0;
    c->is_true = 1;
    c->grow_rho = 0;
    c->hist_cap = 0;
}

// ------------------------------------------------------------------ plan
struct Plan {
    int device = 0;
    int on_device = 0;
    int64_t m = 0, n = 0;
    DevOperand A, At;
    int sms = 0, grid = 0;
    Ctl* ctl = nullptr;          // device control block
    Ctl* stage = nullptr;        // pinned host staging / read-back of the control block
    int32_t* poll = nullptr;     // pinned host, 2 polled status words
    int* flag_dev = nullptr;
    int* flag_host = nullptr;    // pinned
    double* partials = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *tmp_m = nullptr, *tmp_n = nullptr;
    double* z[kTMax] = {};
    double* u[kTMax] = {};
    double *d = nullptr, *c = nullptr, *v = nullptr, *bt = nullptr;
    double *xbest = nullptr, *wx = nullptr, *wd = nullptr;
    double* hist = nullptr;
    int64_t hist_alloc = 0;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // cached graphs of one block of iterations
    cudaGraphExec_t g_cta = nullptr;
    int g_cta_key = -1;
    int64_t g_cta_launches = 0;
    int g_cta_iters = 0;
    cudaGraphExec_t g_ta[3] = {nullptr, nullptr, nullptr};   // plain, normal system, LP (c_+)
    int64_t g_ta_launches[3] = {0, 0, 0};
    int g_ta_iters[3] = {0, 0, 0};
    // mixed precision: FP32 values of A / Aᵀ (structure shared), FP32 chain vectors
    DevCSR32 A32, At32;
    float* z32[kTMax] = {};
    float* u32[kTMax] = {};
    float* r32 = nullptr;
    float* dx32 = nullptr;
    float chain_scale = 1.0f;    // 1/sigma, sigma a power of two >= sqrt(||A||_1 ||A||_inf) >= ||A||_2
    cudaGraphExec_t g_cta32 = nullptr;
    int g_cta32_key = -1;
    int64_t g_cta32_launches = 0;
    int g_cta32_iters = 0;
    // fused chain (A and Aᵀ both run-staged): blocks of the cooperative launch per
    // precision (0: not available) and the per-block moment partials
    int chain_grid = 0, chain_grid32 = 0;
    int dia_grid = 0, dia_grid32 = 0;   // the same on the diagonal form (0: A has none)
    double* chain_part = nullptr;    // (2 kTMax + 4) x the largest of those grids
    int chain_part_grid = 0;         // that grid
    bool fused = false;              // this call runs the fused chain
    bool dia = false;                // ... on the diagonal form
    bool step = false;               // ... as the fused step (auxiliary solve and update in the launch)
    int dc_size = 0;                 // dense A held on chip by a cluster of this many blocks (0: no)
    bool dcl = false;                // this call runs the on-chip dense step
    // opt-in profiling of the iteration's products (events around each launch)
    bool profiling = false;
    int prof_count = 0;
    std::vector<cudaEvent_t> pev;
    size_t pev_used = 0;
    double prof_bytes = 0.0;
};

// algorithmic bytes of one product: stored values and indices, row offsets,
// the input vector read once and the output vector written once
static double spmv_bytes(const DevOperand& A) {
    const double R = (double)A.rows(), C = (double)A.cols();
    if (A.format == TACTA_CSR) return 12.0 * (double)A.csr.nnz + 4.0 * (R + 1.0) + 8.0 * C + 8.0 * R;
    return 8.0 * R * C + 8.0 * C + 8.0 * R;
}

// a product of the iteration chain; timed with a pair of events when profiling
static cudaError_t chain_spmv(Plan* p, const LaunchCtx& L, const DevOperand& A, const double* x, double* y,
                              int epi, EpiArgs e, FinArgs f, int gate) {
    if (!p->profiling) return launch_spmv(L, A, x, y, epi, e, f, gate);
    while (p->pev.size() < p->pev_used + 2) {
        cudaEvent_t ev;
        cudaError_t err = cudaEventCreate(&ev);
        if (err != cudaSuccess) return err;
        p->pev.push_back(ev);
    }
    cudaError_t err = cudaEventRecord(p->pev[p->pev_used], L.stream);
    if (err != cudaSuccess) return err;
    if ((err = launch_spmv(L, A, x, y, epi, e, f, gate)) != cudaSuccess) return err;
    if ((err = cudaEventRecord(p->pev[p->pev_used + 1], L.stream)) != cudaSuccess) return err;
    p->pev_used += 2;
    p->prof_bytes += spmv_bytes(A);
    p->prof_count += 1;
    return cudaSuccess;
}

static void prof_begin(Plan* p, int profile) {
    p->profiling = profile != 0;
    p->pev_used = 0;
    p->prof_bytes = 0.0;
    p->prof_count = 0;
}

static void prof_end(Plan* p, tacta_info* info) {
    if (!info) return;
    if (!p->profiling) return;
    double ms = 0.0;
    for (size_t i = 0; i + 1 < p->pev_used; i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->pev[i], p->pev[i + 1]) == cudaSuccess) ms += t;
    }
    info->spmv_count = p->prof_count;
    info->spmv_ms = ms;
    info->spmv_bytes = p->prof_bytes;
    p->profiling = false;
}

static void free_graphs(Plan* p) {
    if (p->g_cta) cudaGraphExecDestroy(p->g_cta);
    p->g_cta = nullptr;
    p->g_cta_key = -1;
    if (p->g_cta32) cudaGraphExecDestroy(p->g_cta32);
    p->g_cta32 = nullptr;
    p->g_cta32_key = -1;
    for (int i = 0; i < 3; ++i) {
        if (p->g_ta[i]) cudaGraphExecDestroy(p->g_ta[i]);
        p->g_ta[i] = nullptr;
    }
}

static void plan_free(Plan* p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    free_graphs(p);
    auto F = [](void* q) { if (q) cudaFree(q); };
    F(p->A.csr.rowptr); F(p->A.csr.colidx); F(p->A.csr.vals); F(p->A.csr.tiles); F(p->A.csr.xwin); F(p->A.csr.runs); F(p->A.csr.lcol);
    F(p->A.dense.vals);
    F(p->At.csr.rowptr); F(p->At.csr.colidx); F(p->At.csr.vals); F(p->At.csr.tiles); F(p->At.csr.xwin); F(p->At.csr.runs); F(p->At.csr.lcol);
    F(p->At.dense.vals);
    F(p->ctl); F(p->partials); F(p->flag_dev); F(p->chain_part);
    F(p->b); F(p->x); F(p->r); F(p->tmp_m); F(p->tmp_n);
    for (int i = 0; i < kTMax; ++i) { F(p->z[i]); F(p->u[i]); }
    F(p->d); F(p->c); F(p->v); F(p->bt); F(p->xbest); F(p->wx); F(p->wd); F(p->hist);
    F(p->A32.vals); F(p->At32.vals); F(p->r32); F(p->dx32);
    for (DevDIA* d : {&p->A.csr.dia, &p->At.csr.dia}) { F(d->vals); F(d->vals32); F(d->mask); F(d->runs); F(d->sbase); }
    for (int i = 0; i < kTMax; ++i) { F(p->z32[i]); F(p->u32[i]); }
    if (p->stage) cudaFreeHost(p->stage);
    if (p->poll) cudaFreeHost(p->poll);
    if (p->flag_host) cudaFreeHost(p->flag_host);
    if (p->cap) cudaStreamDestroy(p->cap);
    for (int i = 0; i < 2; ++i) if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    for (cudaEvent_t e : p->pev) cudaEventDestroy(e);
    cudaSetDevice(cur);
    delete p;
}

// Kernel choice for a CSR operand: rows averaging >= 64 nonzeros run warp per
// row; shorter rows run the TMA-staged row tiles (one FP64 FMA chain per
// thread, every lane busy), provided no single row exceeds a tile's capacity.
// Tiles: greedy runs of consecutive rows, at most kTileRows rows and `cap`
// nonzeros each, described by {row begin, row end, nnz begin, nnz end}.
// Runs of x for the run-staged product: per tile, the distinct columns (inside the
// tile's window win[t]) split where the gap exceeds kRunGap; each run starts on a column
// that is a multiple of 4 and has a length that is a multiple of 4 (16-byte bulk copies of
// FP64 and of FP32 x), and lcol maps every nonzero to
// its slot in the runs laid end to end. False when a tile needs more than kRunMax runs
// or kRunXs staged entries.
static bool build_runs(const std::vector<int4>& tiles, const std::vector<int2>& win,
                       const std::vector<int32_t>& ci, std::vector<int2>& runs, std::vector<uint16_t>& lcol) {
    runs.assign(tiles.size() * kRunMax, make_int2(0, 0));
    lcol.assign(ci.size() + kPadLcol, 0);
    std::vector<uint8_t> used(kXSpan + 2);
    for (size_t t = 0; t < tiles.size(); ++t) {
        const int z = tiles[t].z, w = tiles[t].w;
        if (w == z) continue;
        const int lo = win[t].x, span = win[t].y - win[t].x + 1;
        std::fill(used.begin(), used.begin() + span, 0);
        for (int k = z; k < w; ++k) used[ci[k] - lo] = 1;
        int2* rt = &runs[t * kRunMax];
        int nrun = 0, total = 0, first = -1, last = -1;
        auto close_run = [&]() {
            if (nrun == kRunMax) return false;
            const int c0 = (lo + first) & ~3;
            const int len = (lo + last + 1 - c0 + 3) & ~3;
            rt[nrun++] = make_int2(c0, len);
            total += len;
            return total <= kRunXs;
        };
        for (int c = 0; c < span; ++c) {
            if (!used[c]) continue;
            if (first >= 0 && c - last > kRunGap) {
                if (!close_run()) return false;
                first = -1;
            }
            if (first < 0) first = c;
            last = c;
        }
        if (!close_run()) return false;
        for (int k = z; k < w; ++k) {
            int off = 0, r = 0;
            while (ci[k] >= rt[r].x + rt[r].y) off += rt[r++].y;
            lcol[k] = (uint16_t)(off + ci[k] - rt[r].x);
        }
    }
    return true;
}

// Device-built run-staged layout (fixed 256-row tiles): true when every tile fits the
// run-staged product; otherwise nothing is kept and the host path decides.
static bool setup_run_tiles_device(DevCSR& a, cudaStream_t s, cudaError_t* err) {
    const int64_t ntiles = (a.rows + kTileRows - 1) / kTileRows;
    int32_t* stats = nullptr;
    int32_t h[4] = {0, 0, 0, 0};
    auto fail = [&](cudaError_t e) {
        cudaFree(a.tiles); cudaFree(a.xwin); cudaFree(a.runs); cudaFree(a.lcol); cudaFree(stats);
        a.tiles = nullptr; a.xwin = nullptr; a.runs = nullptr; a.lcol = nullptr;
        *err = e;
        return false;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&a.tiles, sizeof(int4) * ntiles)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&a.xwin, sizeof(int2) * ntiles)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&a.runs, sizeof(int2) * kRunMax * ntiles)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&a.lcol, sizeof(uint16_t) * (a.nnz + kPadLcol))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&stats, sizeof(int32_t) * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(a.lcol, 0, sizeof(uint16_t) * (a.nnz + kPadLcol), s)) != cudaSuccess) return fail(e);
    if ((e = run_tiles_build(s, a, a.tiles, a.xwin, a.runs, a.lcol, stats)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e);
    if (h[0] != 0 || h[1] > kRunCap || h[2] > kXSpan) return fail(cudaSuccess);
    cudaFree(stats);
    a.ntiles = (int)ntiles;
    a.cap = (h[1] <= kXCapCompactPlan && h[2] <= kXSpanCompactPlan) ? kXCapCompactPlan : kTileCapSmall;
    a.cfg.kind = 3;
    return true;
}

static cudaError_t setup_csr_kernel(DevCSR& a, cudaStream_t s) {
    const double avg = a.rows > 0 ? (double)a.nnz / (double)a.rows : 0.0;
    a.cfg.kind = 1;
    if (avg >= 64.0) return cudaSuccess;
    if (a.nnz > 0 && avg * kTileRows <= (double)kRunCap) {
        cudaError_t e = cudaSuccess;
        if (setup_run_tiles_device(a, s, &e)) return spmv_tiled_prepare();
        if (e != cudaSuccess) return e;
    }
    std::vector<int32_t> rp((size_t)a.rows + 1);
    cudaError_t e = cudaMemcpyAsync(rp.data(), a.rowptr, sizeof(int32_t) * (a.rows + 1), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const int cap = avg * kTileRows <= 0.9 * kTileCapSmall ? kTileCapSmall : kTileCapLarge;
    int32_t maxrow = 0;
    for (int64_t i = 0; i < a.rows; ++i) maxrow = std::max(maxrow, rp[i + 1] - rp[i]);
    if (maxrow > cap) return cudaSuccess;   // an outlier row: keep warp per row
    std::vector<int4> tiles;
    tiles.reserve((size_t)(a.rows / kTileRows + a.nnz / cap + 2));
    int64_t r = 0;
    while (r < a.rows) {
        int64_t e2 = r;
        while (e2 < a.rows && e2 - r < kTileRows && (int64_t)rp[e2 + 1] - rp[r] <= cap) ++e2;
        tiles.push_back(make_int4((int)r, (int)e2, rp[r], rp[e2]));
        r = e2;
    }
    if ((e = cudaMalloc(&a.tiles, sizeof(int4) * tiles.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(a.tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    a.ntiles = (int)tiles.size();
    a.cap = cap;
    a.cfg.kind = 2;
    // banded? every tile's columns within a window of kXSpan entries of x (aligned start)
    if (cap == kTileCapSmall && a.nnz > 0) {
        std::vector<int32_t> ci((size_t)a.nnz);
        if ((e = cudaMemcpyAsync(ci.data(), a.colidx, sizeof(int32_t) * a.nnz, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        std::vector<int2> win(tiles.size());
        bool banded = true;
        for (size_t t = 0; t < tiles.size() && banded; ++t) {
            int lo = INT32_MAX, hi = -1;
            for (int k = tiles[t].z; k < tiles[t].w; ++k) { lo = std::min(lo, ci[k]); hi = std::max(hi, ci[k]); }
            if (hi < 0) { lo = 0; hi = 0; }
            win[t] = make_int2(lo, hi);
            if (hi - (lo & ~1) + 1 > kXSpan) banded = false;
        }
        if (banded) {
            // the compact instance (three blocks per SM) when every tile fits it
            int32_t max_nnz = 0, max_span = 0;
            for (size_t t = 0; t < tiles.size(); ++t) {
                max_nnz = std::max(max_nnz, tiles[t].w - tiles[t].z);
                max_span = std::max(max_span, win[t].y - (win[t].x & ~1) + 1);
            }
            if (max_nnz <= kXCapCompactPlan && max_span <= kXSpanCompactPlan) a.cap = kXCapCompactPlan;
            if ((e = cudaMalloc(&a.xwin, sizeof(int2) * win.size())) != cudaSuccess) return e;
            if ((e = cudaMemcpyAsync(a.xwin, win.data(), sizeof(int2) * win.size(), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess) return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            a.cfg.kind = 3;
            std::vector<int2> runs;
            std::vector<uint16_t> lcol;
            if (max_nnz <= kRunCap && build_runs(tiles, win, ci, runs, lcol)) {
                if ((e = cudaMalloc(&a.runs, sizeof(int2) * runs.size())) != cudaSuccess) return e;
                if ((e = cudaMalloc(&a.lcol, sizeof(uint16_t) * lcol.size())) != cudaSuccess) return e;
                if ((e = cudaMemcpyAsync(a.runs, runs.data(), sizeof(int2) * runs.size(), cudaMemcpyHostToDevice,
                                         s)) != cudaSuccess) return e;
                if ((e = cudaMemcpyAsync(a.lcol, lcol.data(), sizeof(uint16_t) * lcol.size(), cudaMemcpyHostToDevice,
                                         s)) != cudaSuccess) return e;
                if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            }
        }
    }
    return spmv_tiled_prepare();
}

static tacta_status validate_opts(const tacta_options& o) {
    if (!(std::isfinite(o.tol) && o.tol > 0.0)) { set_error("tol must be finite and > 0"); return TACTA_ERR_INVALID; }
    if (!std::isfinite(o.tol_normal)) { set_error("tol_normal must be finite"); return TACTA_ERR_INVALID; }
    if (o.t_max < 1 || o.t_max > kTMax) { set_error("t_max must be in 1..8"); return TACTA_ERR_INVALID; }
    if (o.max_iter < 0) { set_error("max_iter must be >= 0"); return TACTA_ERR_INVALID; }
    if (o.recompute_every < 0) { set_error("recompute_every must be >= 0"); return TACTA_ERR_INVALID; }
    if (o.cycle < 0 || o.cycle > 2) { set_error("unknown cycle"); return TACTA_ERR_INVALID; }
    if (o.fused_chain < 0 || o.fused_chain > 3) { set_error("fused_chain must be in 0..3"); return TACTA_ERR_INVALID; }
    if (o.wait_limit_log2 < 0 || o.wait_limit_log2 > 40) {
        set_error("wait_limit_log2 must be in 0..40");
        return TACTA_ERR_INVALID;
    }
    if (o.precision != TACTA_PRECISION_FP64 && o.precision != TACTA_PRECISION_MIXED) {
        set_error("unknown precision");
        return TACTA_ERR_INVALID;
    }
    return TACTA_OK;
}

static tacta_status plan_create(const tacta_matrix* M, const tacta_options* opt, Plan** out) {
    *out = nullptr;
    if (!M) { set_error("A is NULL"); return TACTA_ERR_INVALID; }
    if (M->m < 1 || M->n < 1) { set_error("A must have m >= 1 and n >= 1"); return TACTA_ERR_INVALID; }
    if (M->m >= (1LL << 31) || M->n >= (1LL << 31)) { set_error("m and n must be < 2^31"); return TACTA_ERR_INVALID; }
    if (M->format != TACTA_DENSE && M->format != TACTA_CSR) { set_error("unknown format"); return TACTA_ERR_INVALID; }
    if (!M->vals && (M->format == TACTA_DENSE || M->nnz > 0)) { set_error("A.vals is NULL"); return TACTA_ERR_INVALID; }
    if (M->format == TACTA_DENSE && M->m * M->n > (1LL << 40)) { set_error("dense A too large"); return TACTA_ERR_INVALID; }
    if (M->format == TACTA_CSR) {
        if (!M->rowptr || (M->nnz > 0 && !M->colidx)) { set_error("CSR arrays missing"); return TACTA_ERR_INVALID; }
        if (M->nnz < 0 || M->nnz >= (1LL << 31)) { set_error("nnz must be in [0, 2^31)"); return TACTA_ERR_INVALID; }
    }
    Plan* p = new Plan();
    p->on_device = M->on_device ? 1 : 0;
    p->m = M->m;
    p->n = M->n;
    cudaStream_t s = opt && opt->stream ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    auto fail = [&](tacta_status st) { plan_free(p); return st; };
#define PTRY(expr)                                                                        \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                \
            return fail(e_ == cudaErrorMemoryAllocation ? TACTA_ERR_OOM : TACTA_ERR_CUDA); \
        }                                                                                 \
    } while (0)
    PTRY(cudaGetDevice(&p->device));
    PTRY(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device));
    p->grid = p->sms * 8;
    PTRY(cudaMallocHost(&p->flag_host, sizeof(int)));
    PTRY(cudaMalloc(&p->flag_dev, sizeof(int)));
    const int64_t m = p->m, n = p->n;
    if (M->format == TACTA_CSR) {
        const int64_t nnz = M->nnz;
        DevCSR& a = p->A.csr;
        p->A.format = p->At.format = TACTA_CSR;
        a.rows = m; a.cols = n; a.nnz = nnz;
        PTRY(cudaMalloc(&a.rowptr, sizeof(int32_t) * (m + 1 + kPadRowptr)));
        PTRY(cudaMalloc(&a.colidx, sizeof(int32_t) * (nnz + kPadColidx)));
        PTRY(cudaMalloc(&a.vals, sizeof(double) * (nnz + kPadVals)));
        PTRY(cudaMemsetAsync(a.rowptr, 0, sizeof(int32_t) * (m + 1 + kPadRowptr), s));
        PTRY(cudaMemsetAsync(a.colidx, 0, sizeof(int32_t) * (nnz + kPadColidx), s));
        PTRY(cudaMemsetAsync(a.vals, 0, sizeof(double) * (nnz + kPadVals), s));
        PTRY(cudaMemcpyAsync(a.rowptr, M->rowptr, sizeof(int32_t) * (m + 1), cudaMemcpyDefault, s));
        if (nnz > 0) {
            PTRY(cudaMemcpyAsync(a.colidx, M->colidx, sizeof(int32_t) * nnz, cudaMemcpyDefault, s));
            PTRY(cudaMemcpyAsync(a.vals, M->vals, sizeof(double) * nnz, cudaMemcpyDefault, s));
        }
        PTRY(csr_validate(s, a.rowptr, a.colidx, m, n, nnz, p->flag_dev, p->flag_host));
        if (*p->flag_host) {
            const int f = *p->flag_host;
            std::string msg = "invalid CSR structure:";
            if (f & 1) msg += " rowptr[0] != 0;";
            if (f & 2) msg += " rowptr decreases;";
            if (f & 4) msg += " rowptr[m] != nnz;";
            if (f & 8) msg += " column index out of range;";
            set_error(msg);
            return fail(TACTA_ERR_INVALID);
        }
        PTRY(csr_transpose(s, a, p->At.csr));
        PTRY(setup_csr_kernel(a, s));
        PTRY(setup_csr_kernel(p->At.csr, s));
        const DevCSR& at = p->At.csr;
        if (a.cfg.kind == 3 && a.lcol && at.cfg.kind == 3 && at.lcol) {
            const int tiles = std::max(a.ntiles, at.ntiles);
            p->chain_grid = cta_chain_grid(p->sms, tiles, false, false);
            p->chain_grid32 = cta_chain_grid(p->sms, tiles, true, false);
            // the diagonal form, when both A and Aᵀ have one (banded with few diagonals)
            PTRY(dia_build(s, a, a.dia, p->flag_dev, p->flag_host));
            if (a.dia.k > 0) PTRY(dia_build(s, p->At.csr, p->At.csr.dia, p->flag_dev, p->flag_host));
            if (a.dia.k > 0 && p->At.csr.dia.k == a.dia.k) {
                const int dt = std::max(a.dia.ntiles, p->At.csr.dia.ntiles);
                p->dia_grid = cta_chain_grid(p->sms, dt, false, true);
                p->dia_grid32 = cta_chain_grid(p->sms, dt, true, true);
            }
            const int g = std::max(std::max(p->chain_grid, p->chain_grid32), std::max(p->dia_grid, p->dia_grid32));
            // 2t products' partials, the fused step's true-residual partials (2 rows) and
            // its ||r||² partials (2 per block)
            if (g > 0) PTRY(cudaMalloc(&p->chain_part, sizeof(double) * (2 * kTMax + 4) * g));
            p->chain_part_grid = g;
        }
    } else {
        p->A.format = p->At.format = TACTA_DENSE;
        DevDense& a = p->A.dense;
        DevDense& t = p->At.dense;
        a.rows = m; a.cols = n; t.rows = n; t.cols = m;
        PTRY(cudaMalloc(&a.vals, sizeof(double) * m * n));
        PTRY(cudaMalloc(&t.vals, sizeof(double) * m * n));
        PTRY(cudaMemcpyAsync(a.vals, M->vals, sizeof(double) * m * n, cudaMemcpyDefault, s));
        PTRY(dense_transpose(s, a.vals, m, n, t.vals));
        a.cfg.kind = n >= 64 ? 1 : 0;
        t.cfg.kind = m >= 64 ? 1 : 0;
        p->dc_size = dense_cluster_size(m, n);   // small enough to keep on chip in one cluster
    }
    const int64_t mn = std::max(m, n);
    PTRY(cudaMalloc(&p->ctl, sizeof(Ctl)));
    PTRY(cudaMemsetAsync(p->ctl, 0, sizeof(Ctl), s));
    PTRY(cudaMallocHost(&p->stage, sizeof(Ctl)));
    PTRY(cudaMallocHost(&p->poll, 2 * sizeof(int32_t)));
    PTRY(cudaMalloc(&p->partials, sizeof(double) * 2 * p->grid));
    // every vector that a product may read carries kPadVec doubles of zeroed padding
    auto vec = [&](double** ptr, int64_t len) {
        cudaError_t e2 = cudaMalloc(ptr, sizeof(double) * (len + kPadVec));
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(*ptr, 0, sizeof(double) * (len + kPadVec), s);
        return e2;
    };
    PTRY(vec(&p->b, m));
    PTRY(vec(&p->x, n));
    PTRY(vec(&p->r, m));
    PTRY(vec(&p->tmp_m, m));
    PTRY(vec(&p->tmp_n, n));
    PTRY(vec(&p->d, mn));
    PTRY(vec(&p->c, n));
    PTRY(vec(&p->v, mn));
    PTRY(vec(&p->bt, n));
    PTRY(vec(&p->xbest, n));
    PTRY(vec(&p->wx, n));
    PTRY(vec(&p->wd, mn));
    PTRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) PTRY(cudaEventCreateWithFlags(&p->ev[i], cudaEventDisableTiming));
    PTRY(cudaStreamSynchronize(s));
#undef PTRY
    *out = p;
    return TACTA_OK;
}

static tacta_status ensure_chain(Plan* p, int t_max) {
    for (int i = 0; i < t_max; ++i) {
        if (!p->z[i]) {
            free_graphs(p);
            CUDA_TRY(cudaMalloc(&p->z[i], sizeof(double) * (p->n + kPadVec)));
            CUDA_TRY(cudaMalloc(&p->u[i], sizeof(double) * (p->m + kPadVec)));
            CUDA_TRY(cudaMemset(p->z[i], 0, sizeof(double) * (p->n + kPadVec)));
            CUDA_TRY(cudaMemset(p->u[i], 0, sizeof(double) * (p->m + kPadVec)));
        }
    }
    return TACTA_OK;
}

static tacta_status ensure_hist(Plan* p, int64_t cap) {
    if (cap <= p->hist_alloc) return TACTA_OK;
    free_graphs(p);  // graphs hold the history pointer
    if (p->hist) cudaFree(p->hist);
    p->hist = nullptr;
    p->hist_alloc = 0;
    CUDA_TRY(cudaMalloc(&p->hist, sizeof(double) * cap));
    p->hist_alloc = cap;
    return TACTA_OK;
}

// FP32 copies and vectors of the mixed-precision path (made on first use)
static tacta_status ensure_mixed(Plan* p, int t_max, cudaStream_t s) {
    auto f32 = [&](float** ptr, int64_t len) {
        cudaError_t e = cudaMalloc(ptr, sizeof(float) * (len + kPadVec32));
        if (e == cudaSuccess) e = cudaMemsetAsync(*ptr, 0, sizeof(float) * (len + kPadVec32), s);
        return e;
    };
    // chain scale 1/sigma from the infinity norms of A and Aᵀ (see below)
    auto set_scale = [&](double ninf, double n1) {
        const double bound = std::sqrt(ninf * n1);
        int e2 = 0;
        if (bound > 0.0 && std::isfinite(bound)) e2 = (int)std::ceil(std::log2(bound));
        e2 = std::max(-120, std::min(120, e2));
        p->chain_scale = std::ldexp(1.0f, -e2);
    };
    if (p->A.format == TACTA_DENSE && !p->A32.vals) {
        // dense A: FP32 copies of A and Aᵀ (row-major), read by the dense FP32 products
        free_graphs(p);
        const int64_t mn = p->m * p->n;
        CUDA_TRY(cudaMalloc(&p->A32.vals, sizeof(float) * (mn + kPadVals32)));
        CUDA_TRY(cudaMalloc(&p->At32.vals, sizeof(float) * (mn + kPadVals32)));
        if (mn > 0) {
            CUDA_TRY(convert_to_f32(s, p->A.dense.vals, p->A32.vals, mn));
            CUDA_TRY(convert_to_f32(s, p->At.dense.vals, p->At32.vals, mn));
        }
        CUDA_TRY(f32(&p->r32, p->m));
        CUDA_TRY(f32(&p->dx32, p->n));
        CUDA_TRY(dense32_prepare());
        CUDA_TRY(dense_abs_row_sum_max(s, p->m, p->n, p->A.dense.vals, p->partials, &p->stage->red[0]));
        const double ninf = p->stage->red[0];
        CUDA_TRY(dense_abs_row_sum_max(s, p->n, p->m, p->At.dense.vals, p->partials, &p->stage->red[0]));
        set_scale(ninf, p->stage->red[0]);
    }
    if (p->A.format == TACTA_CSR && !p->A32.vals) {
        free_graphs(p);
        for (DevCSR32* a : {&p->A32, &p->At32}) {
            const DevCSR& base = (a == &p->A32) ? p->A.csr : p->At.csr;
            a->base = &base;
            CUDA_TRY(cudaMalloc(&a->vals, sizeof(float) * (base.nnz + kPadVals32)));
            CUDA_TRY(cudaMemsetAsync(a->vals, 0, sizeof(float) * (base.nnz + kPadVals32), s));
            if (base.nnz > 0) CUDA_TRY(convert_to_f32(s, base.vals, a->vals, base.nnz));
        }
        CUDA_TRY(f32(&p->r32, p->m));
        CUDA_TRY(f32(&p->dx32, p->n));
        for (DevDIA* d : {&p->A.csr.dia, &p->At.csr.dia}) {
            if (d->k == 0) continue;
            const int64_t nv = (int64_t)d->ntiles * d->k * kTileRows;
            CUDA_TRY(cudaMalloc(&d->vals32, sizeof(float) * nv));
            CUDA_TRY(convert_to_f32(s, d->vals, d->vals32, nv));
        }
        CUDA_TRY(spmv32_prepare());
        // chain scale: products are multiplied by 1/sigma so the FP32 chain vectors stay
        // within range (H^i r grows like ||A||^(2i)); sigma is a power of two (exact)
        double ninf = 0.0, n1 = 0.0;
        CUDA_TRY(abs_row_sum_max(s, p->A.csr, p->partials, &p->stage->red[0]));
        ninf = p->stage->red[0];
        CUDA_TRY(abs_row_sum_max(s, p->At.csr, p->partials, &p->stage->red[0]));
        n1 = p->stage->red[0];
        set_scale(ninf, n1);
    }
    for (int i = 0; i < t_max; ++i) {
        if (!p->z32[i]) {
            free_graphs(p);
            CUDA_TRY(f32(&p->z32[i], p->n));
            CUDA_TRY(f32(&p->u32[i], p->m));
        }
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    return TACTA_OK;
}

template <typename V>
static ChainOps<V> chain_ops(const DevCSR& At, const DevCSR& A, const V* at_vals, const V* a_vals) {
    ChainOps<V> o;
    const DevCSR* op[2] = {&At, &A};
    for (int i = 0; i < 2; ++i) {
        o.tiles[i] = op[i]->tiles;
        o.runs[i] = op[i]->runs;
        o.rowptr[i] = op[i]->rowptr;
        o.lcol[i] = op[i]->lcol;
        o.ntiles[i] = op[i]->ntiles;
    }
    o.vals[0] = at_vals;
    o.vals[1] = a_vals;
    return o;
}

template <typename V>
static ChainOpsDia<V> chain_ops_dia(const DevCSR& At, const DevCSR& A, const V* at_vals, const V* a_vals) {
    ChainOpsDia<V> o;
    const DevCSR* op[2] = {&At, &A};
    for (int i = 0; i < 2; ++i) {
        o.mask[i] = op[i]->dia.mask;
        o.runs[i] = op[i]->dia.runs;
        o.sbase[i] = op[i]->dia.sbase;
        o.ntiles[i] = op[i]->dia.ntiles;
        o.rows[i] = (int)op[i]->rows;
    }
    o.vals[0] = at_vals;
    o.vals[1] = a_vals;
    o.k = A.dia.k;
    return o;
}

// algorithmic bytes of one product on the diagonal form: the tiles' values (k per row,
// zeros where a row lacks a diagonal) and row masks, x read once, y written once
static double dia_bytes(const DevCSR& a, double vsize) {
    const double rows_t = (double)a.dia.ntiles * kTileRows;
    return vsize * (double)a.dia.k * rows_t + rows_t + vsize * (double)a.cols + vsize * (double)a.rows;
}

// events around the fused chain when profiling: it counts as its 2t products
static cudaError_t prof_mark(Plan* p, const LaunchCtx& L) {
    if (!p->profiling) return cudaSuccess;
    while (p->pev.size() < p->pev_used + 1) {
        cudaEvent_t ev;
        cudaError_t err = cudaEventCreate(&ev);
        if (err != cudaSuccess) return err;
        p->pev.push_back(ev);
    }
    return cudaEventRecord(p->pev[p->pev_used++], L.stream);
}

// One F_t step, mixed precision: FP32 chain and update, then (gated on the device)
// the refinement: fold the FP32 correction into the FP64 x and recompute the true
// residual b - A x with the FP64 product, stored back into the FP32 residual.
static cudaError_t chain_spmv32(Plan* p, const LaunchCtx& L, const DevCSR32& A, const float* x, float* y,
                                FinArgs f) {
    const bool dense = p->A.format == TACTA_DENSE;
    const bool tr = &A == &p->At32;                       // the product with Aᵀ (n x m)
    auto launch = [&]() {
        return dense ? launch_dense32(L, tr ? p->n : p->m, tr ? p->m : p->n, A.vals, x, y, p->chain_scale, f,
                                      GATE_ALWAYS)
                     : launch_spmv32(L, A, x, y, p->chain_scale, EPI_NORM, f, GATE_ALWAYS);
    };
    if (!p->profiling) return launch();
    while (p->pev.size() < p->pev_used + 2) {
        cudaEvent_t ev;
        cudaError_t err = cudaEventCreate(&ev);
        if (err != cudaSuccess) return err;
        p->pev.push_back(ev);
    }
    cudaError_t err = cudaEventRecord(p->pev[p->pev_used], L.stream);
    if (err != cudaSuccess) return err;
    if ((err = launch()) != cudaSuccess) return err;
    if ((err = cudaEventRecord(p->pev[p->pev_used + 1], L.stream)) != cudaSuccess) return err;
    p->pev_used += 2;
    p->prof_count += 1;
    if (dense) {   // the FP32 values once, x read and y written once
        p->prof_bytes += 4.0 * (double)(p->m * p->n) + 4.0 * (double)(p->m + p->n);
    } else {
        const DevCSR& a = *A.base;
        p->prof_bytes += 8.0 * (double)a.nnz + 4.0 * (double)(a.rows + 1) + 4.0 * (double)a.cols +
                         4.0 * (double)a.rows;
    }
    return cudaSuccess;
}

// algorithmic bytes of one CTA F_t step of order t on CSR operands, unfused: t products
// with Aᵀ and t with A (values and column indices, row offsets), the chain's vectors read
// and written once per product, and the update reading t z's, t u's and x, r and writing
// x, r; vsize = 8 (FP64) or 4 (the FP32 chain: FP32 values and vectors)
static double fpt_bytes(const Plan* p, int t, double vsize) {
    const double m = (double)p->m, n = (double)p->n, nnz = (double)p->A.nnz();
    const double ba = (vsize + 4.0) * nnz + 4.0 * (m + 1.0), bat = (vsize + 4.0) * nnz + 4.0 * (n + 1.0);
    return t * (ba + bat) + vsize * t * (m + 2.0 * n + m) + vsize * (t + 2.0) * (n + m);
}

static cudaError_t enqueue_cta32_iter(Plan* p, const LaunchCtx& L, int t) {
    cudaError_t e;
    if (p->fused) {
        ChainVecs<float> v;
        v.r = p->r32;
        for (int i = 0; i < kTMax; ++i) { v.z[i] = p->z32[i]; v.u[i] = p->u32[i]; }
        if ((e = prof_mark(p, L)) != cudaSuccess) return e;
        if (p->dia) {
            e = launch_cta_chain_dia32(L, chain_ops_dia<float>(p->At.csr, p->A.csr, p->At.csr.dia.vals32,
                                                               p->A.csr.dia.vals32),
                                       v, t, p->chain_scale, p->chain_part, p->dia_grid32, nullptr);
        } else {
            e = launch_cta_chain32(L, chain_ops<float>(p->At.csr, p->A.csr, p->At32.vals, p->A32.vals), v, t,
                                   p->chain_scale, p->chain_part, p->chain_grid32, nullptr);
        }
        if (e != cudaSuccess) return e;
        if ((e = prof_mark(p, L)) != cudaSuccess) return e;
        if (p->profiling) {
            for (const DevCSR* a : {&p->At.csr, &p->A.csr})
                p->prof_bytes += t * (p->dia ? dia_bytes(*a, 4.0)
                                             : 8.0 * (double)a->nnz + 4.0 * (double)(a->rows + 1) +
                                                   4.0 * (double)a->cols + 4.0 * (double)a->rows);
            p->prof_count += 2 * t;
        }
        if ((e = launch_cta_aux_step(L, t, p->chain_part, p->dia ? p->dia_grid32 : p->chain_grid32)) !=
            cudaSuccess) return e;
    } else {
        const float* uprev = p->r32;
        for (int i = 0; i < t; ++i) {
            if ((e = chain_spmv32(p, L, p->At32, uprev, p->z32[i], FinArgs{FIN_PHI, 2 * i + 1, nullptr})) !=
                cudaSuccess) return e;
            if ((e = chain_spmv32(p, L, p->A32, p->z32[i], p->u32[i], FinArgs{FIN_PHI, 2 * i + 2, nullptr})) !=
                cudaSuccess) return e;
            uprev = p->u32[i];
        }
        if ((e = launch_cta_aux_step(L, t)) != cudaSuccess) return e;
    }
    if ((e = launch_cta_update32(L, t, p->m, p->n, p->dx32, p->r32, p->z32, p->u32, p->chain_scale,
                                 FinArgs{FIN_CTA_UPDATE, 0, p->hist})) != cudaSuccess) return e;
    if ((e = launch_fold_correction(L, p->n, p->x, p->dx32, GATE_NEED_TRUE)) != cudaSuccess) return e;
    return launch_spmv(L, p->A, p->x, p->tmp_m, EPI_RESID_F32, EpiArgs{p->b, nullptr, p->r32},
                       FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE);
}

// ------------------------------------------------------------------ options

struct Opts {
    tacta_options o;
    cudaStream_t s;
};

static Opts resolve(const tacta_options* opt) {
    Opts r;
    tacta_default_options(&r.o);
    if (opt) r.o = *opt;
    if (r.o.tol_normal < 0.0) r.o.tol_normal = r.o.tol;
    if (!(r.o.tol_cta > 0.0)) r.o.tol_cta = r.o.tol;
    if (!(r.o.pivot_tol > 0.0)) r.o.pivot_tol = r.o.precision == TACTA_PRECISION_MIXED ? 1e-6 : 1e-12;
    if (r.o.poll_every < 1) r.o.poll_every = 64;
    r.s = (cudaStream_t)r.o.stream;
    return r;
}

static int schedule(int64_t k, int t_max, int cycle) {
    if (cycle == TACTA_CYCLE_FIXED || t_max == 1) return t_max;
    if (cycle == TACTA_CYCLE_SAWTOOTH) return 1 + (int)(k % t_max);
    const int period = 2 * t_max - 2;
    const int j = (int)(k % period);
    return j < t_max ? j + 1 : 2 * t_max - 1 - j;
}

static int schedule_period(int t_max, int cycle) {
    if (cycle == TACTA_CYCLE_FIXED || t_max == 1) return 1;
    if (cycle == TACTA_CYCLE_SAWTOOTH) return t_max;
    return 2 * t_max - 2;
}

// ------------------------------------------------------------------ iteration bodies

static cudaError_t enqueue_cta_iter(Plan* p, const LaunchCtx& L, int t) {
    cudaError_t e;
    if (p->fused) {
        ChainVecs<double> v;
        v.r = p->r;
        for (int i = 0; i < kTMax; ++i) { v.z[i] = p->z[i]; v.u[i] = p->u[i]; }
        if ((e = prof_mark(p, L)) != cudaSuccess) return e;
        if (p->dia) {
            e = launch_cta_chain_dia(L, chain_ops_dia<double>(p->At.csr, p->A.csr, p->At.csr.dia.vals,
                                                              p->A.csr.dia.vals),
                                     v, t, p->chain_part, p->dia_grid, nullptr);
        } else {
            e = launch_cta_chain(L, chain_ops<double>(p->At.csr, p->A.csr, p->At.csr.vals, p->A.csr.vals), v, t,
                                 p->chain_part, p->chain_grid, nullptr);
        }
        if (e != cudaSuccess) return e;
        if ((e = prof_mark(p, L)) != cudaSuccess) return e;
        if (p->profiling) {
            p->prof_bytes += t * (p->dia ? dia_bytes(p->At.csr, 8.0) + dia_bytes(p->A.csr, 8.0)
                                         : spmv_bytes(p->At) + spmv_bytes(p->A));
            p->prof_count += 2 * t;
        }
        if ((e = launch_cta_aux_step(L, t, p->chain_part, p->dia ? p->dia_grid : p->chain_grid)) != cudaSuccess)
            return e;
        if ((e = launch_cta_update(L, t, p->m, p->n, p->x, p->r, p->z, p->u,
                                   FinArgs{FIN_CTA_UPDATE, 0, p->hist})) != cudaSuccess) return e;
        return launch_spmv(L, p->A, p->x, p->r, EPI_RESID, EpiArgs{p->b, nullptr, nullptr},
                           FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE);
    }
    const double* uprev = p->r;
    EpiArgs none{nullptr, nullptr, nullptr};
    for (int i = 0; i < t; ++i) {
        if ((e = chain_spmv(p, L, p->At, uprev, p->z[i], EPI_NORM, none, FinArgs{FIN_PHI, 2 * i + 1, nullptr},
                            GATE_ALWAYS)) != cudaSuccess) return e;
        if ((e = chain_spmv(p, L, p->A, p->z[i], p->u[i], EPI_NORM, none, FinArgs{FIN_PHI, 2 * i + 2, nullptr},
                            GATE_ALWAYS)) != cudaSuccess) return e;
        uprev = p->u[i];
    }
    if ((e = launch_cta_aux_step(L, t)) != cudaSuccess) return e;
    if ((e = launch_cta_update(L, t, p->m, p->n, p->x, p->r, p->z, p->u,
                               FinArgs{FIN_CTA_UPDATE, 0, p->hist})) != cudaSuccess) return e;
    return launch_spmv(L, p->A, p->x, p->r, EPI_RESID, EpiArgs{p->b, nullptr, nullptr},
                       FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE);
}

// Up to nsteps F_t steps in one persistent launch of the fused step (the order of each
// step follows the cycle from the device's step count). FP64: a true residual a step asks
// for runs as the first product of the next step. FP32 chain: the launch ends early when a
// refinement is due, which the two gated launches after it carry out (fold the FP32
// correction into the FP64 x, FP64 residual b - A x).
static cudaError_t enqueue_cta_steps(Plan* p, const LaunchCtx& L, int nsteps, int t_max, int cycle, bool mixed) {
    cudaError_t e;
    if ((e = prof_mark(p, L)) != cudaSuccess) return e;
    if (!mixed) {
        ChainVecs<double> v;
        v.r = p->r;
        for (int i = 0; i < kTMax; ++i) { v.z[i] = p->z[i]; v.u[i] = p->u[i]; }
        StepArgs<double> sa;
        sa.x = p->x;
        sa.r = p->r;
        sa.m = p->m;
        sa.n = p->n;
        sa.hist = p->hist;
        sa.rpart = p->chain_part + (size_t)2 * kTMax * p->chain_part_grid;
        sa.upart = p->chain_part + (size_t)(2 * kTMax + 2) * p->chain_part_grid;
        sa.b = p->b;
        sa.nsteps = nsteps;
        sa.t_max = t_max;
        sa.cycle = cycle;
        if (p->dia)
            e = launch_cta_chain_dia(L, chain_ops_dia<double>(p->At.csr, p->A.csr, p->At.csr.dia.vals,
                                                              p->A.csr.dia.vals),
                                     v, 0, p->chain_part, p->dia_grid, &sa);
        else
            e = launch_cta_chain(L, chain_ops<double>(p->At.csr, p->A.csr, p->At.csr.vals, p->A.csr.vals), v, 0,
                                 p->chain_part, p->chain_grid, &sa);
        if (e != cudaSuccess) return e;
        return prof_mark(p, L);
    }
    ChainVecs<float> v;
    v.r = p->r32;
    for (int i = 0; i < kTMax; ++i) { v.z[i] = p->z32[i]; v.u[i] = p->u32[i]; }
    StepArgs<float> sa;
    sa.x = p->dx32;
    sa.r = p->r32;
    sa.m = p->m;
    sa.n = p->n;
    sa.xscale = p->chain_scale;
    sa.hist = p->hist;
    sa.upart = p->chain_part + (size_t)(2 * kTMax + 2) * p->chain_part_grid;
    sa.nsteps = nsteps;
    sa.t_max = t_max;
    sa.cycle = cycle;
    if (p->dia)
        e = launch_cta_chain_dia32(L, chain_ops_dia<float>(p->At.csr, p->A.csr, p->At.csr.dia.vals32,
                                                           p->A.csr.dia.vals32),
                                   v, 0, p->chain_scale, p->chain_part, p->dia_grid32, &sa);
    else
        e = launch_cta_chain32(L, chain_ops<float>(p->At.csr, p->A.csr, p->At32.vals, p->A32.vals), v, 0,
                               p->chain_scale, p->chain_part, p->chain_grid32, &sa);
    if (e != cudaSuccess) return e;
    if ((e = prof_mark(p, L)) != cudaSuccess) return e;
    if ((e = launch_fold_correction(L, p->n, p->x, p->dx32, GATE_NEED_TRUE)) != cudaSuccess) return e;
    return launch_spmv(L, p->A, p->x, p->tmp_m, EPI_RESID_F32, EpiArgs{p->b, nullptr, p->r32},
                       FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE);
}

// operator of TA: M = A (normal = 0) or M = AᵀA (normal = 1), rhs = b or Aᵀb
static cudaError_t apply_M(Plan* p, const LaunchCtx& L, int normal, const double* in, double* out,
                           int epi, EpiArgs e, FinArgs f, int gate) {
    if (!normal) return launch_spmv(L, p->A, in, out, epi, e, f, gate);
    cudaError_t err = launch_spmv(L, p->A, in, p->tmp_m, EPI_NONE, EpiArgs{nullptr, nullptr, nullptr},
                                  FinArgs{FIN_NONE, 0, nullptr}, gate);
    if (err != cudaSuccess) return err;
    return launch_spmv(L, p->At, p->tmp_m, out, epi, e, f, gate);
}
static cudaError_t apply_Mt(Plan* p, const LaunchCtx& L, int normal, const double* in, double* out,
                            int epi, EpiArgs e, FinArgs f, int gate) {
    if (!normal) return launch_spmv(L, p->At, in, out, epi, e, f, gate);
    return apply_M(p, L, 1, in, out, epi, e, f, gate);   // AᵀA is symmetric
}

static cudaError_t enqueue_ta_iter(Plan* p, const LaunchCtx& L, int normal, int nonneg, double* hist) {
    cudaError_t e;
    const double* rhs = normal ? p->bt : p->b;
    const int64_t mm = normal ? p->n : p->m;
    EpiArgs none{nullptr, nullptr, nullptr};
    // c = Mᵀ (b - b') (c_+ = max(c, 0) for LP feasibility), ||c||², pivot test (Eq. eqlem2) / rho growth
    if (!normal) {
        if ((e = chain_spmv(p, L, p->At, p->d, p->c, nonneg ? EPI_NORM_POS : EPI_NORM, none,
                            FinArgs{FIN_TA_C, 0, nullptr}, GATE_ALWAYS)) != cudaSuccess) return e;
    } else if ((e = apply_Mt(p, L, normal, p->d, p->c, EPI_NORM, none, FinArgs{FIN_TA_C, 0, nullptr},
                             GATE_ALWAYS)) != cudaSuccess) return e;
    // v = rho M c / ||c|| (Eq. vr) with the dots of Eq. alph
    if ((e = apply_M(p, L, normal, p->c, p->v, EPI_TAPIVOT, EpiArgs{rhs, p->d, nullptr},
                     FinArgs{FIN_TA_V, 0, nullptr}, GATE_PIVOT)) != cudaSuccess) return e;
    if ((e = launch_ta_update(L, mm, p->n, p->x, p->d, rhs, p->v, p->c,
                              FinArgs{FIN_TA_UPDATE, 0, hist})) != cudaSuccess) return e;
    return apply_M(p, L, normal, p->x, p->d, EPI_RESID, EpiArgs{rhs, nullptr, nullptr},
                   FinArgs{FIN_TRUE_RES, 0, hist}, GATE_NEED_TRUE);
}

// ------------------------------------------------------------------ iteration loop with polling

struct LoopResult { int64_t launches = 0; };

// Runs iterations until the device stop flag is set or max_iter iterations were enqueued.
// body(L, k) enqueues iteration k; graph holds a captured block of `gper` iterations (optional).
template <class Body>
static tacta_status run_loop(Plan* p, const Opts& O, int64_t max_iter, int period, bool use_graph,
                             cudaGraphExec_t* graph, int64_t* graph_launches, int* graph_iters,
                             Body body, int64_t* launches) {
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, launches};
    if (max_iter <= 0) return TACTA_OK;
    const int64_t poll = std::max<int64_t>(O.o.poll_every, 1);
    if (use_graph) {
        // The iteration loop on the device: one graph whose WHILE node repeats a body of
        // ceil(poll / period) schedule periods of iterations followed by loop_continue,
        // which keeps the node running while the control block's status is 0 and the
        // body count is below the bound that covers max_iter; no host polling, and no
        // launches enqueued past the stop.
        const int reps = (int)std::max<int64_t>(1, (poll + period - 1) / period);
        const int iters = reps * period;
        if (*graph == nullptr) {
            int64_t cnt = 0;
            LaunchCtx C{p->cap, p->ctl, p->partials, p->grid, &cnt};
            cudaGraph_t g = nullptr;
            cudaGraphConditionalHandle h = 0;
            CUDA_TRY(cudaGraphCreate(&g, 0));
            cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
            cudaGraphNodeParams np{};
            cudaGraphNode_t node = nullptr;
            if (e == cudaSuccess) {
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = h;
                np.conditional.type = cudaGraphCondTypeWhile;
                np.conditional.size = 1;
                e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
            }
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(p->cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int k = 0; k < iters && e == cudaSuccess; ++k) e = body(C, (int64_t)k);
                if (e == cudaSuccess) e = launch_loop_continue(p->cap, p->ctl, h);
                cudaGraph_t captured = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(p->cap, &captured);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                *graph = nullptr;
                set_error(std::string("graph with the on-device loop: ") + cudaGetErrorString(e));
                return TACTA_ERR_CUDA;
            }
            *graph_launches = cnt + 1;   // the body's kernels and loop_continue
            *graph_iters = iters;
        }
        const int64_t limit = (max_iter + iters - 1) / iters;
        CUDA_TRY(launch_loop_begin(O.s, p->ctl, (int32_t)std::min<int64_t>(limit, INT32_MAX)));
        CUDA_TRY(cudaGraphLaunch(*graph, O.s));
        // bodies run, for the launch count
        CUDA_TRY(cudaMemcpyAsync(&p->poll[0], &p->ctl->loops, sizeof(int32_t), cudaMemcpyDeviceToHost, O.s));
        CUDA_TRY(cudaStreamSynchronize(O.s));
        *launches += 1 + (int64_t)p->poll[0] * *graph_launches;
        return TACTA_OK;
    }
    if (use_graph && *graph == nullptr) {
        // capture ceil(poll / period) periods of iterations on the private stream
        const int reps = (int)std::max<int64_t>(1, (poll + period - 1) / period);
        const int iters = reps * period;
        int64_t cnt = 0;
        LaunchCtx C{p->cap, p->ctl, p->partials, p->grid, &cnt};
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < iters && e == cudaSuccess; ++k) e = body(C, (int64_t)k);
        cudaError_t e2 = cudaStreamEndCapture(p->cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            set_error(std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
            return TACTA_ERR_CUDA;
        }
        e = cudaGraphInstantiate(graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            *graph = nullptr;
            set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
            return TACTA_ERR_CUDA;
        }
        *graph_launches = cnt;
        *graph_iters = iters;
    }
    int64_t k = 0;
    int chunk = 0;
    bool stopped = false;
    while (k < max_iter && !stopped) {
        if (use_graph) {
            CUDA_TRY(cudaGraphLaunch(*graph, O.s));
            *launches += *graph_launches;
            k += *graph_iters;
        } else {
            const int64_t todo = std::min<int64_t>(poll, max_iter - k);
            for (int64_t j = 0; j < todo; ++j) CUDA_TRY(body(L, k + j));
            k += todo;
        }
        const int slot = chunk & 1;
        CUDA_TRY(cudaMemcpyAsync(&p->poll[slot], &p->ctl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, O.s));
        CUDA_TRY(cudaEventRecord(p->ev[slot], O.s));
        if (p->profiling) {   // profiled runs poll without lag: no gated launches in the timings
            CUDA_TRY(cudaEventSynchronize(p->ev[slot]));
            if (p->poll[slot] != 0) stopped = true;
        } else if (chunk > 0) {
            CUDA_TRY(cudaEventSynchronize(p->ev[slot ^ 1]));
            if (p->poll[slot ^ 1] != 0) stopped = true;
        }
        ++chunk;
    }
    return TACTA_OK;
}

// ------------------------------------------------------------------ shared bits

static tacta_status read_ctl(Plan* p, cudaStream_t s) {
    CUDA_TRY(cudaMemcpyAsync(p->stage, p->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return TACTA_OK;
}

static tacta_status write_ctl(Plan* p, cudaStream_t s, const Ctl& h) {
    // the staging buffer is reused: wait for earlier users of the stream first
    CUDA_TRY(cudaStreamSynchronize(s));
    *p->stage = h;
    CUDA_TRY(cudaMemcpyAsync(p->ctl, p->stage, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    return TACTA_OK;
}

static tacta_status status_of(int reason) {
    switch (reason) {
    case TACTA_REASON_RESIDUAL:
    case TACTA_REASON_NORMAL:
    case TACTA_REASON_GAP:
    case TACTA_REASON_ZERO_RHS:
    case TACTA_REASON_RHO_BOUND:
    case TACTA_REASON_ENHANCED: return TACTA_OK;
    case TACTA_REASON_TIMEOUT: return TACTA_ERR_TIMEOUT;
    case TACTA_REASON_MAXITER: return TACTA_MAXITER;
    case TACTA_REASON_BREAKDOWN: return TACTA_BREAKDOWN;
    case TACTA_REASON_WITNESS: return TACTA_WITNESS;
    case TACTA_REASON_NONFINITE: return TACTA_ERR_NONFINITE;
    default: return TACTA_MAXITER;
    }
}

// true ||b - A x||² and ||Aᵀ(b - A x)||² at exit, into ctl->red[0], ctl->red[2]
static tacta_status exit_residuals(Plan* p, const Opts& O, const double* x, int64_t* launches) {
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, launches};
    CUDA_TRY(launch_spmv(L, p->A, x, p->tmp_m, EPI_RESID, EpiArgs{p->b, nullptr, nullptr},
                         FinArgs{FIN_STORE, 0, nullptr}, GATE_FORCE));
    CUDA_TRY(launch_spmv(L, p->At, p->tmp_m, p->tmp_n, EPI_NORM, EpiArgs{nullptr, nullptr, nullptr},
                         FinArgs{FIN_STORE, 2, nullptr}, GATE_FORCE));
    return TACTA_OK;
}

static Ctl base_ctl(const Opts& O, int64_t hist_cap) {
    Ctl h;
    std::memset(&h, 0, sizeof(h));
    h.max_iter = O.o.max_iter;
    h.R = O.o.recompute_every;
    h.hist_cap = (int32_t)hist_cap;
    h.tol2 = O.o.tol * O.o.tol;
    h.cs2 = 1.0;
    h.rho_max = O.o.rho_max > 0.0 ? O.o.rho_max : INFINITY;
    h.tol_n2 = O.o.tol_normal * O.o.tol_normal;
    h.pivot_tol = O.o.pivot_tol;
    h.wait_cycles = 1LL << (O.o.wait_limit_log2 > 0 ? O.o.wait_limit_log2 : 31);
    return h;
}

struct VecIO {   // caller vectors
    const double* b;
    const double* x0;
    double* x_out;
    double* hist;
    int32_t hist_cap;
};

static tacta_status load_b(Plan* p, const Opts& O, const VecIO& io) {
    if (!io.b) { set_error("b is NULL"); return TACTA_ERR_INVALID; }
    if (!io.x_out) { set_error("x_out is NULL"); return TACTA_ERR_INVALID; }
    CUDA_TRY(cudaMemcpyAsync(p->b, io.b, sizeof(double) * p->m, cudaMemcpyDefault, O.s));
    return TACTA_OK;
}

static tacta_status store_out(Plan* p, const Opts& O, const VecIO& io, const double* x, int hist_len,
                              int64_t* launches = nullptr) {
    CUDA_TRY(cudaMemcpyAsync(io.x_out, x, sizeof(double) * p->n, cudaMemcpyDefault, O.s));
    if (io.hist && io.hist_cap > 0 && hist_len > 0) {
        const int64_t h = std::min<int64_t>(hist_len, io.hist_cap);
        CUDA_TRY(launch_hist_sqrt(O.s, p->hist, h));
        if (launches) ++*launches;
        CUDA_TRY(cudaMemcpyAsync(io.hist, p->hist, sizeof(double) * h, cudaMemcpyDefault, O.s));
    }
    CUDA_TRY(cudaStreamSynchronize(O.s));
    return TACTA_OK;
}

// ------------------------------------------------------------------ CTA (Alg. 1.1)

// Runs CTA from x0 (or 0) on the plan's b; leaves x in p->x and the final control block in p->stage.
static tacta_status cta_core(Plan* p, const Opts& O, const double* x0, int64_t hist_cap, int64_t* launches) {
    tacta_status st;
    const bool mixed = O.o.precision == TACTA_PRECISION_MIXED;
    if (mixed && (st = ensure_mixed(p, O.o.t_max, O.s)) != TACTA_OK) return st;
    if (!mixed && (st = ensure_chain(p, O.o.t_max)) != TACTA_OK) return st;
    if ((st = ensure_hist(p, std::max<int64_t>(hist_cap, 1))) != TACTA_OK) return st;
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, launches};
    Ctl h = base_ctl(O, hist_cap);
    h.need_true = (x0 || mixed) ? 1 : 0;
    h.enhanced = (!mixed && O.o.enhanced) ? 1 : 0;
    if (mixed) {
        h.cs2 = (double)p->chain_scale * (double)p->chain_scale;
        h.ref_eta2 = kRefineEta2;
    }
    if ((st = write_ctl(p, O.s, h)) != TACTA_OK) return st;
    EpiArgs none{nullptr, nullptr, nullptr};
    CUDA_TRY(launch_reduce_vec(L, p->m, p->b, nullptr, FinArgs{FIN_SETUP_B, 0, nullptr}, GATE_ALWAYS));
    CUDA_TRY(launch_spmv(L, p->At, p->b, p->tmp_n, EPI_NORM, none, FinArgs{FIN_SETUP_MTB, 0, nullptr}, GATE_ALWAYS));
    if (mixed) {
        if (x0) CUDA_TRY(cudaMemcpyAsync(p->x, x0, sizeof(double) * p->n, cudaMemcpyDefault, O.s));
        else CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
        CUDA_TRY(cudaMemsetAsync(p->dx32, 0, sizeof(float) * p->n, O.s));
        CUDA_TRY(launch_spmv(L, p->A, p->x, p->tmp_m, EPI_RESID_F32, EpiArgs{p->b, nullptr, p->r32},
                             FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE));
    } else if (x0) {
        CUDA_TRY(cudaMemcpyAsync(p->x, x0, sizeof(double) * p->n, cudaMemcpyDefault, O.s));
        CUDA_TRY(launch_spmv(L, p->A, p->x, p->r, EPI_RESID, EpiArgs{p->b, nullptr, nullptr},
                             FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE));
    } else {
        CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
        CUDA_TRY(cudaMemcpyAsync(p->r, p->b, sizeof(double) * p->m, cudaMemcpyDeviceToDevice, O.s));
        CUDA_TRY(launch_reduce_vec(L, p->m, p->r, nullptr, FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_ALWAYS));
    }
    const int t_max = O.o.t_max, cycle = O.o.cycle;
    const int period = schedule_period(t_max, cycle);
    p->dia = (O.o.fused_chain == 1 || O.o.fused_chain == 3) && (mixed ? p->dia_grid32 : p->dia_grid) > 0;
    p->fused = p->dia || (O.o.fused_chain != 0 && (mixed ? p->chain_grid32 : p->chain_grid) > 0);
    p->step = p->fused && O.o.fused_chain != 3;
    p->dcl = !mixed && p->A.format == TACTA_DENSE && p->dc_size > 0 && O.o.fused_chain != 0;
    const int nsteps = std::max(1, O.o.poll_every);   // F_t steps per launch of the fused step
    const int key = ((((t_max * 4 + cycle) * 4 + (p->fused ? 1 : 0) + (p->dia ? 2 : 0)) * 2 + (p->step ? 1 : 0)) * 2 +
                     (p->dcl ? 1 : 0)) * 4096 + std::min(nsteps, 4095);
    cudaGraphExec_t* g = mixed ? &p->g_cta32 : &p->g_cta;
    int* gkey = mixed ? &p->g_cta32_key : &p->g_cta_key;
    if (*g && *gkey != key) {
        cudaGraphExecDestroy(*g);
        *g = nullptr;
    }
    *gkey = key;
    if (p->dcl) {
        // small dense A on chip: one cluster launch runs up to nsteps steps; the device stops at max_iter
        Opts O1 = O;
        O1.o.poll_every = 1;
        const int64_t calls = ((int64_t)O.o.max_iter + nsteps - 1) / nsteps + 8;
        auto body = [&](const LaunchCtx& LL, int64_t) {
            cudaError_t e = prof_mark(p, LL);
            if (e != cudaSuccess) return e;
            DenseClusterArgs a{p->A.dense.vals, p->At.dense.vals, p->m, p->n, p->x, p->r, p->b, p->hist,
                               nsteps, t_max, cycle};
            if ((e = launch_cta_dense_cluster(LL, a, p->dc_size)) != cudaSuccess) return e;
            return prof_mark(p, LL);
        };
        st = run_loop(p, O1, calls, 1, O.o.use_graph != 0, g, &p->g_cta_launches, &p->g_cta_iters, body, launches);
    } else if (p->step) {
        // one body = one launch of up to nsteps steps; the device stops at max_iter. FP64
        // launches run their nsteps unless the solve stops; an FP32-chain launch may end
        // early for a refinement, so up to one launch per step may be needed
        Opts O1 = O;
        O1.o.poll_every = 1;
        // (a few spare launches: a pass whose chain is dropped for a true residual does
        // not count as a step)
        const int64_t calls = mixed ? (int64_t)O.o.max_iter + 1 : ((int64_t)O.o.max_iter + nsteps - 1) / nsteps + 8;
        auto body = [&](const LaunchCtx& LL, int64_t) { return enqueue_cta_steps(p, LL, nsteps, t_max, cycle, mixed); };
        st = run_loop(p, O1, calls, 1, O.o.use_graph != 0, g, mixed ? &p->g_cta32_launches : &p->g_cta_launches,
                      mixed ? &p->g_cta32_iters : &p->g_cta_iters, body, launches);
    } else {
        auto body = [&](const LaunchCtx& LL, int64_t k) {
            const int t = schedule(k, t_max, cycle);
            return mixed ? enqueue_cta32_iter(p, LL, t) : enqueue_cta_iter(p, LL, t);
        };
        st = run_loop(p, O, O.o.max_iter, period, O.o.use_graph != 0, g,
                      mixed ? &p->g_cta32_launches : &p->g_cta_launches,
                      mixed ? &p->g_cta32_iters : &p->g_cta_iters, body, launches);
    }
    if (st != TACTA_OK) return st;
    // the FP64 fused step runs a pending true residual at the start of the next step: after
    // the last step it runs here (a no-op when none is pending or the solve has stopped)
    if (!mixed && (p->step || p->dcl))
        CUDA_TRY(launch_spmv(L, p->A, p->x, p->r, EPI_RESID, EpiArgs{p->b, nullptr, nullptr},
                             FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE));
    if (mixed) CUDA_TRY(launch_fold_correction(L, p->n, p->x, p->dx32, GATE_FORCE));
    CUDA_TRY(cudaGetLastError());
    return TACTA_OK;
}

static void fill_info(tacta_info* info, const Ctl& c, tacta_status st, int64_t launches) {
    if (!info) return;
    std::memset(info, 0, sizeof(*info));
    info->status = st;
    info->reason = c.status;
    info->iters = c.k;
    info->matvecs = c.matvecs;
    info->rel_res = c.bn2 > 0 ? std::sqrt(c.red[0] / c.bn2) : 0.0;
    info->rel_normal_res = c.mtbn2 > 0 ? std::sqrt(c.red[2] / c.mtbn2) : 0.0;
    info->rho = c.rho;
    info->hist_len = c.hist_len;
    info->launches = launches;
}

static tacta_status plan_cta(Plan* p, const VecIO& io, const tacta_options* opt, tacta_info* info) {
    Opts O = resolve(opt);
    tacta_status st;
    if ((st = validate_opts(O.o)) != TACTA_OK) return st;
    CUDA_TRY(cudaSetDevice(p->device));
    if ((st = load_b(p, O, io)) != TACTA_OK) return st;
    int64_t launches = 0;
    const int64_t hist_cap = io.hist && io.hist_cap > 0 ? std::min<int64_t>(io.hist_cap, (int64_t)O.o.max_iter + 1) : 0;
    if (O.o.profile) O.o.use_graph = 0;
    prof_begin(p, O.o.profile);
    if ((st = cta_core(p, O, io.x0, hist_cap, &launches)) != TACTA_OK) { p->profiling = false; return st; }
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    if (p->profiling && (p->step || p->dcl)) {   // the timed unit is an F_t step: the launches ran stage->k of them
        const bool mixed = O.o.precision == TACTA_PRECISION_MIXED;
        p->prof_count = p->stage->k;
        p->prof_bytes = 0.0;
        for (int k = 0; k < p->stage->k; ++k)
            p->prof_bytes += fpt_bytes(p, schedule(k, O.o.t_max, O.o.cycle), mixed ? 4.0 : 8.0);
    }
    if (p->stage->status == TACTA_REASON_ZERO_RHS) CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
    if ((st = exit_residuals(p, O, p->x, &launches)) != TACTA_OK) return st;
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    Ctl c = *p->stage;
    if ((st = store_out(p, O, io, p->x, c.hist_len, &launches)) != TACTA_OK) return st;
    const tacta_status out = status_of(c.status);
    if (out == TACTA_ERR_NONFINITE) set_error("non-finite value in a reduction");
    fill_info(info, c, out, launches);
    prof_end(p, info);
    p->profiling = false;
    if (info && c.status == TACTA_REASON_ZERO_RHS) { info->rel_res = 0.0; info->rel_normal_res = 0.0; }
    return out;
}

// ------------------------------------------------------------------ TA (Alg. 2.2 / 2.1)

// Starts TA on M (normal: AᵀA with rhs Aᵀb) from (x, d) already in p->x / p->d.
static tacta_status ta_setup(Plan* p, const Opts& O, int normal, const double* x0, int64_t hist_cap,
                             int64_t* launches) {
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, launches};
    const double* rhs = normal ? p->bt : p->b;
    const int64_t mm = normal ? p->n : p->m;
    EpiArgs none{nullptr, nullptr, nullptr};
    CUDA_TRY(launch_reduce_vec(L, mm, rhs, nullptr, FinArgs{FIN_SETUP_B, 0, nullptr}, GATE_ALWAYS));
    CUDA_TRY(apply_Mt(p, L, normal, rhs, p->tmp_n, EPI_NORM, none, FinArgs{FIN_SETUP_MTB, 0, nullptr}, GATE_ALWAYS));
    if (x0) {
        CUDA_TRY(cudaMemcpyAsync(p->x, x0, sizeof(double) * p->n, cudaMemcpyDefault, O.s));
        CUDA_TRY(launch_reduce_vec(L, p->n, p->x, nullptr, FinArgs{FIN_SETUP_RHO, 0, nullptr}, GATE_ALWAYS));
        CUDA_TRY(apply_M(p, L, normal, p->x, p->d, EPI_RESID, EpiArgs{rhs, nullptr, nullptr},
                         FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_NEED_TRUE));
    } else {
        CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
        CUDA_TRY(cudaMemcpyAsync(p->d, rhs, sizeof(double) * mm, cudaMemcpyDeviceToDevice, O.s));
        CUDA_TRY(launch_reduce_vec(L, mm, p->d, rhs, FinArgs{FIN_TRUE_RES, 0, p->hist}, GATE_ALWAYS));
    }
    (void)hist_cap;
    return TACTA_OK;
}

// TA iterations; the history pointer is always the plan's buffer (trips of Alg. 2.5 run with
// hist_cap = 0 in the control block, so they write no history and share the cached graph).
static tacta_status ta_iterate(Plan* p, const Opts& O, int normal, int64_t max_iter, int64_t* launches) {
    const int nonneg = (!normal && O.o.nonneg) ? 1 : 0;
    const int slot = nonneg ? 2 : normal;
    auto body = [&](const LaunchCtx& LL, int64_t) { return enqueue_ta_iter(p, LL, normal, nonneg, p->hist); };
    return run_loop(p, O, max_iter, 1, O.o.use_graph != 0, &p->g_ta[slot], &p->g_ta_launches[slot],
                    &p->g_ta_iters[slot], body, launches);
}

static tacta_status plan_ta(Plan* p, const VecIO& io, const tacta_options* opt, tacta_info* info) {
    Opts O = resolve(opt);
    tacta_status st;
    if ((st = validate_opts(O.o)) != TACTA_OK) return st;
    CUDA_TRY(cudaSetDevice(p->device));
    if ((st = load_b(p, O, io)) != TACTA_OK) return st;
    int64_t launches = 0;
    const int64_t hist_cap = io.hist && io.hist_cap > 0 ? std::min<int64_t>(io.hist_cap, (int64_t)O.o.max_iter + 1) : 0;
    if ((st = ensure_hist(p, std::max<int64_t>(hist_cap, 1))) != TACTA_OK) return st;
    Ctl h = base_ctl(O, hist_cap);
    h.grow_rho = 1;
    h.nonneg = O.o.nonneg ? 1 : 0;
    h.need_true = io.x0 ? 1 : 0;
    if ((st = write_ctl(p, O.s, h)) != TACTA_OK) return st;
    if ((st = ta_setup(p, O, 0, io.x0, hist_cap, &launches)) != TACTA_OK) return st;
    if (O.o.profile) O.o.use_graph = 0;
    prof_begin(p, O.o.profile);
    if ((st = ta_iterate(p, O, 0, O.o.max_iter, &launches)) != TACTA_OK) { p->profiling = false; return st; }
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    if (p->stage->status == TACTA_REASON_ZERO_RHS) CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
    if ((st = exit_residuals(p, O, p->x, &launches)) != TACTA_OK) return st;
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    Ctl c = *p->stage;
    if ((st = store_out(p, O, io, p->x, c.hist_len, &launches)) != TACTA_OK) return st;
    const tacta_status out = status_of(c.status);
    if (out == TACTA_ERR_NONFINITE) set_error("non-finite value in a reduction");
    if (out == TACTA_ERR_TIMEOUT) set_error("a bounded wait inside a kernel gave up");
    fill_info(info, c, out, launches);
    prof_end(p, info);
    p->profiling = false;
    if (info && c.status == TACTA_REASON_ZERO_RHS) { info->rel_res = 0.0; info->rel_normal_res = 0.0; }
    return out;
}

// ------------------------------------------------------------------ hybrid minimum norm (Sec. 5.2, Alg. 2.5)

struct BisectOut {
    double rho_hi = 0.0, rho_lo = 0.0;
    int64_t used = 0;     // TA iterations over all trips
    int trips = 0;
    int reason = TACTA_REASON_GAP;
};

// Algorithm 2.5 (Sec. 4.4) on M x = rhs, M = A (normal = 0) or AᵀA with rhs = Aᵀb
// (normal = 1), from the approximate solution x_eps held in p->x (b already loaded).
// rho_hi = ||x_eps||, rho_lo = 0; while rho_hi - rho_lo > tol ||x_eps||: rho = the midpoint,
// Alg. 2.1 at rho from the last witness (from 0 before the first), on success
// rho_hi = rho and its x is the answer, on a witness rho_lo = (b - b')ᵀb / ||Mᵀ(b - b')||
// (Cor. cor1). A normal-equation stop of a trip ends the call with that x. The answer is
// left in p->xbest. With trip_log non-null, trip i writes 6 doubles at trip_log[6 i]:
// rho, the trip's stop reason, rho_hi and rho_lo after the trip, its iterations, 0.
static tacta_status minnorm_bisect(Plan* p, const Opts& O, int normal, double* trip_log, int log_cap,
                                   int64_t* launches, BisectOut* out) {
    tacta_status st;
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, launches};
    EpiArgs none{nullptr, nullptr, nullptr};
    if (normal)
        CUDA_TRY(launch_spmv(L, p->At, p->b, p->bt, EPI_NONE, none, FinArgs{FIN_NONE, 0, nullptr}, GATE_FORCE));
    CUDA_TRY(cudaMemcpyAsync(p->xbest, p->x, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, O.s));
    Ctl h = base_ctl(O, 0);
    if ((st = write_ctl(p, O.s, h)) != TACTA_OK) return st;
    CUDA_TRY(launch_reduce_vec(L, p->n, p->x, nullptr, FinArgs{FIN_STORE, 0, nullptr}, GATE_ALWAYS));
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    double rho_hi = std::sqrt(p->stage->red[0]);
    double rho_lo = 0.0;
    const double gap = O.o.tol * rho_hi;
    // thresholds of the operator in use (||rhs||², ||Mᵀ rhs||²)
    const double* rhs = normal ? p->bt : p->b;
    const int64_t mm = normal ? p->n : p->m;
    CUDA_TRY(launch_reduce_vec(L, mm, rhs, nullptr, FinArgs{FIN_SETUP_B, 0, nullptr}, GATE_ALWAYS));
    CUDA_TRY(apply_Mt(p, L, normal, rhs, p->tmp_n, EPI_NORM, none, FinArgs{FIN_SETUP_MTB, 0, nullptr}, GATE_ALWAYS));
    bool have_witness = false;
    int64_t used = 0;
    int trips = 0;
    int final_reason = TACTA_REASON_GAP;
    while (rho_hi - rho_lo > gap) {
        if (used >= O.o.max_iter) { final_reason = TACTA_REASON_MAXITER; break; }
        const double rho = 0.5 * (rho_hi + rho_lo);
        ctl_set_trip<<<1, 1, 0, O.s>>>(p->ctl, rho, (int)(O.o.max_iter - used));
        ++*launches;
        CUDA_TRY(cudaGetLastError());
        if (have_witness) {
            CUDA_TRY(cudaMemcpyAsync(p->x, p->wx, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, O.s));
            CUDA_TRY(cudaMemcpyAsync(p->d, p->wd, sizeof(double) * mm, cudaMemcpyDeviceToDevice, O.s));
        } else {
            CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
            CUDA_TRY(cudaMemcpyAsync(p->d, rhs, sizeof(double) * mm, cudaMemcpyDeviceToDevice, O.s));
        }
        CUDA_TRY(launch_reduce_vec(L, mm, p->d, rhs, FinArgs{FIN_TRIP_START, 0, nullptr}, GATE_FORCE));
        if ((st = ta_iterate(p, O, normal, O.o.max_iter - used, launches)) != TACTA_OK) return st;
        if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
        const Ctl c = *p->stage;
        used += c.k;
        bool stop = false;
        if (c.status == TACTA_REASON_RESIDUAL) {
            rho_hi = rho;
            CUDA_TRY(cudaMemcpyAsync(p->xbest, p->x, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, O.s));
        } else if (c.status == TACTA_REASON_WITNESS) {
            rho_lo = c.db / std::sqrt(c.cn2);
            have_witness = true;
            CUDA_TRY(cudaMemcpyAsync(p->wx, p->x, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, O.s));
            CUDA_TRY(cudaMemcpyAsync(p->wd, p->d, sizeof(double) * mm, cudaMemcpyDeviceToDevice, O.s));
        } else if (c.status == TACTA_REASON_NORMAL) {
            CUDA_TRY(cudaMemcpyAsync(p->xbest, p->x, sizeof(double) * p->n, cudaMemcpyDeviceToDevice, O.s));
            final_reason = TACTA_REASON_NORMAL;
            stop = true;
        } else {
            final_reason = c.status;
            stop = true;
        }
        if (trip_log && trips < log_cap) {
            double* row = trip_log + 6 * (size_t)trips;
            row[0] = rho;
            row[1] = (double)c.status;
            row[2] = rho_hi;
            row[3] = rho_lo;
            row[4] = (double)c.k;
            row[5] = 0.0;
        }
        ++trips;
        if (stop) break;
    }
    out->rho_hi = rho_hi;
    out->rho_lo = rho_lo;
    out->used = used;
    out->trips = trips;
    out->reason = final_reason;
    return TACTA_OK;
}

static tacta_status plan_minnorm(Plan* p, const VecIO& io, const tacta_options* opt, tacta_info* info) {
    Opts O = resolve(opt);
    tacta_status st;
    if ((st = validate_opts(O.o)) != TACTA_OK) return st;
    CUDA_TRY(cudaSetDevice(p->device));
    if ((st = load_b(p, O, io)) != TACTA_OK) return st;
    int64_t launches = 0;
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, &launches};
    // phase 1: CTA to tol_cta from x = 0
    Opts Oc = O;
    Oc.o.tol = O.o.tol_cta;
    const int64_t hist_cap = io.hist && io.hist_cap > 0 ? std::min<int64_t>(io.hist_cap, (int64_t)O.o.max_iter + 1) : 0;
    if ((st = cta_core(p, Oc, nullptr, hist_cap, &launches)) != TACTA_OK) return st;
    if ((st = exit_residuals(p, O, p->x, &launches)) != TACTA_OK) return st;
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    const Ctl c1 = *p->stage;
    tacta_info out_info;
    std::memset(&out_info, 0, sizeof(out_info));
    out_info.cta_iters = c1.k;
    out_info.hist_len = c1.hist_len;
    const double bn2_orig = c1.bn2, atbn2_orig = c1.mtbn2;
    if (c1.status == TACTA_REASON_ZERO_RHS) {
        CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
        if ((st = store_out(p, O, io, p->x, c1.hist_len, &launches)) != TACTA_OK) return st;
        out_info.status = TACTA_OK;
        out_info.reason = TACTA_REASON_ZERO_RHS;
        out_info.launches = launches;
        if (info) *info = out_info;
        return TACTA_OK;
    }
    if (status_of(c1.status) != TACTA_OK) {   // CTA did not reach tol_cta
        if ((st = store_out(p, O, io, p->x, c1.hist_len, &launches)) != TACTA_OK) return st;
        const tacta_status s1 = status_of(c1.status);
        fill_info(info, c1, s1, launches);
        if (info) { info->cta_iters = c1.k; info->iters = 0; info->rho = 0.0; info->matvecs = 0; }
        return s1;
    }
    const double rel_res = std::sqrt(c1.red[0] / c1.bn2);
    const int normal = rel_res <= O.o.tol_cta ? 0 : 1;
    // phase 2: Algorithm 2.5 on (A, b) or (AᵀA, Aᵀb) from CTA's x
    BisectOut bo;
    if ((st = minnorm_bisect(p, O, normal, nullptr, 0, &launches, &bo)) != TACTA_OK) return st;
    const double rho_hi = bo.rho_hi, rho_lo = bo.rho_lo;
    const int64_t used = bo.used;
    const int trips = bo.trips;
    const int final_reason = bo.reason;
    // residuals of the original system at x_best
    if ((st = exit_residuals(p, O, p->xbest, &launches)) != TACTA_OK) return st;
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    const Ctl c = *p->stage;
    if ((st = store_out(p, O, io, p->xbest, 0)) != TACTA_OK) return st;
    if (io.hist && io.hist_cap > 0 && c1.hist_len > 0) {
        // the CTA phase history was overwritten only if hist was reused: it was not (trips pass NULL)
        CUDA_TRY(launch_hist_sqrt(O.s, p->hist, std::min<int64_t>(c1.hist_len, io.hist_cap)));
        CUDA_TRY(cudaMemcpyAsync(io.hist, p->hist, sizeof(double) * std::min<int64_t>(c1.hist_len, io.hist_cap),
                                 cudaMemcpyDefault, O.s));
        CUDA_TRY(cudaStreamSynchronize(O.s));
    }
    const tacta_status out = status_of(final_reason);
    if (out == TACTA_ERR_NONFINITE) set_error("non-finite value in a reduction");
    out_info.status = out;
    out_info.reason = final_reason;
    out_info.iters = (int32_t)used;
    out_info.rel_res = std::sqrt(c.red[0] / bn2_orig);
    out_info.rel_normal_res = atbn2_orig > 0 ? std::sqrt(c.red[2] / atbn2_orig) : 0.0;
    out_info.rho = rho_hi;
    out_info.rho_lower = rho_lo;
    out_info.trips = trips;
    out_info.normal_system = normal;
    out_info.launches = launches;
    if (info) *info = out_info;
    return out;
}

// Algorithm 2.5 alone from a caller's approximate solution x_eps of M x = rhs (see
// minnorm_bisect), with the per-trip log on the host.
static tacta_status plan_bisect(Plan* p, const double* b, const double* x_eps, int normal, const tacta_options* opt,
                                double* x_out, double* trip_log, int log_cap, tacta_info* info) {
    Opts O = resolve(opt);
    tacta_status st;
    if ((st = validate_opts(O.o)) != TACTA_OK) return st;
    if (!x_eps) { set_error("x_eps is NULL"); return TACTA_ERR_INVALID; }
    if (normal != 0 && normal != 1) { set_error("normal must be 0 or 1"); return TACTA_ERR_INVALID; }
    if (log_cap < 0 || (log_cap > 0 && !trip_log)) { set_error("trip_log / log_cap"); return TACTA_ERR_INVALID; }
    CUDA_TRY(cudaSetDevice(p->device));
    VecIO io{b, x_eps, x_out, nullptr, 0};
    if ((st = load_b(p, O, io)) != TACTA_OK) return st;
    if ((st = ensure_hist(p, 1)) != TACTA_OK) return st;
    int64_t launches = 0;
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, &launches};
    EpiArgs none{nullptr, nullptr, nullptr};
    // ||b||² and ||Aᵀb||² of the original system, for the exit residuals
    if ((st = write_ctl(p, O.s, base_ctl(O, 0))) != TACTA_OK) return st;
    CUDA_TRY(launch_reduce_vec(L, p->m, p->b, nullptr, FinArgs{FIN_SETUP_B, 0, nullptr}, GATE_FORCE));
    CUDA_TRY(launch_spmv(L, p->At, p->b, p->tmp_n, EPI_NORM, none, FinArgs{FIN_SETUP_MTB, 0, nullptr}, GATE_FORCE));
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    const double bn2 = p->stage->bn2, atbn2 = p->stage->mtbn2;
    tacta_info out_info;
    std::memset(&out_info, 0, sizeof(out_info));
    if (bn2 == 0.0) {
        CUDA_TRY(cudaMemsetAsync(p->x, 0, sizeof(double) * p->n, O.s));
        if ((st = store_out(p, O, io, p->x, 0)) != TACTA_OK) return st;
        out_info.reason = TACTA_REASON_ZERO_RHS;
        if (info) *info = out_info;
        return TACTA_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(p->x, x_eps, sizeof(double) * p->n, cudaMemcpyDefault, O.s));
    BisectOut bo;
    if ((st = minnorm_bisect(p, O, normal, trip_log, log_cap, &launches, &bo)) != TACTA_OK) return st;
    if ((st = exit_residuals(p, O, p->xbest, &launches)) != TACTA_OK) return st;
    if ((st = read_ctl(p, O.s)) != TACTA_OK) return st;
    const Ctl c = *p->stage;
    if ((st = store_out(p, O, io, p->xbest, 0)) != TACTA_OK) return st;
    const tacta_status out = status_of(bo.reason);
    if (out == TACTA_ERR_NONFINITE) set_error("non-finite value in a reduction");
    if (out == TACTA_ERR_TIMEOUT) set_error("a bounded wait inside a kernel gave up");
    out_info.status = out;
    out_info.reason = bo.reason;
    out_info.iters = (int32_t)bo.used;
    out_info.rel_res = std::sqrt(c.red[0] / bn2);
    out_info.rel_normal_res = atbn2 > 0 ? std::sqrt(c.red[2] / atbn2) : 0.0;
    out_info.rho = bo.rho_hi;
    out_info.rho_lower = bo.rho_lo;
    out_info.trips = bo.trips;
    out_info.normal_system = normal;
    out_info.launches = launches;
    if (info) *info = out_info;
    return out;
}

}  // namespace tacta

// ==================================================================== C ABI
using namespace tacta;

struct tacta_plan_s { Plan* p; };

extern "C" {

void tacta_default_options(tacta_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-10;
    o->tol_normal = -1.0;
    o->tol_cta = 0.0;
    o->pivot_tol = 1e-12;
    o->max_iter = 1000;
    o->t_max = 5;
    o->cycle = TACTA_CYCLE_PINGPONG;
    o->recompute_every = 40;
    o->use_graph = 1;
    o->poll_every = 64;
    o->profile = 0;
    o->precision = TACTA_PRECISION_FP64;
    o->nonneg = 0;
    o->fused_chain = 1;
    o->rho_max = 0.0;
    o->stream = nullptr;
}

const char* tacta_last_error(void) { return get_error(); }

int32_t tacta_version(void) { return 10000; }

tacta_status tacta_plan_create(const tacta_matrix* A, const tacta_options* opt, tacta_plan* plan) {
    set_error("");
    if (!plan) { set_error("plan is NULL"); return TACTA_ERR_INVALID; }
    *plan = nullptr;
    Plan* p = nullptr;
    tacta_status st = plan_create(A, opt, &p);
    if (st != TACTA_OK) return st;
    *plan = new tacta_plan_s{p};
    return TACTA_OK;
}

void tacta_plan_destroy(tacta_plan plan) {
    if (!plan) return;
    plan_free(plan->p);
    delete plan;
}

static tacta_status plan_call(int algo, tacta_plan plan, const double* b, const double* x0,
                              const tacta_options* opt, double* x_out, double* hist, int32_t hist_cap,
                              tacta_info* info) {
    set_error("");
    if (!plan || !plan->p) { set_error("plan is NULL"); return TACTA_ERR_INVALID; }
    if (hist_cap < 0) { set_error("hist_cap must be >= 0"); return TACTA_ERR_INVALID; }
    VecIO io{b, x0, x_out, hist, hist_cap};
    if (algo == 0) return plan_cta(plan->p, io, opt, info);
    if (algo == 1) return plan_ta(plan->p, io, opt, info);
    return plan_minnorm(plan->p, io, opt, info);
}

tacta_status tacta_plan_cta(tacta_plan plan, const double* b, const double* x0, const tacta_options* opt,
                            double* x_out, double* hist, int32_t hist_cap, tacta_info* info) {
    return plan_call(0, plan, b, x0, opt, x_out, hist, hist_cap, info);
}
tacta_status tacta_plan_ta(tacta_plan plan, const double* b, const double* x0, const tacta_options* opt,
                           double* x_out, double* hist, int32_t hist_cap, tacta_info* info) {
    return plan_call(1, plan, b, x0, opt, x_out, hist, hist_cap, info);
}
tacta_status tacta_plan_minnorm(tacta_plan plan, const double* b, const double* x0, const tacta_options* opt,
                                double* x_out, double* hist, int32_t hist_cap, tacta_info* info) {
    return plan_call(2, plan, b, x0, opt, x_out, hist, hist_cap, info);
}

tacta_status tacta_plan_minnorm_bisect(tacta_plan plan, const double* b, const double* x_eps, int32_t normal,
                                       const tacta_options* opt, double* x_out, double* trip_log, int32_t log_cap,
                                       tacta_info* info) {
    set_error("");
    if (!plan || !plan->p) { set_error("plan is NULL"); return TACTA_ERR_INVALID; }
    return plan_bisect(plan->p, b, x_eps, normal, opt, x_out, trip_log, log_cap, info);
}

tacta_status tacta_plan_transpose(tacta_plan plan, const tacta_options* opt, tacta_plan* out) {
    set_error("");
    if (!plan || !plan->p || !out) { set_error("NULL argument"); return TACTA_ERR_INVALID; }
    Plan* p = plan->p;
    CUDA_TRY(cudaSetDevice(p->device));
    tacta_matrix M;
    std::memset(&M, 0, sizeof(M));
    M.m = p->n;
    M.n = p->m;
    M.on_device = 1;
    if (p->At.format == TACTA_CSR) {
        M.format = TACTA_CSR;
        M.nnz = p->At.csr.nnz;
        M.vals = p->At.csr.vals;
        M.rowptr = p->At.csr.rowptr;
        M.colidx = p->At.csr.colidx;
    } else {
        M.format = TACTA_DENSE;
        M.vals = p->At.dense.vals;
    }
    Plan* q = nullptr;
    tacta_status st = plan_create(&M, opt, &q);
    if (st != TACTA_OK) return st;
    q->on_device = p->on_device;
    *out = new tacta_plan_s{q};
    return TACTA_OK;
}

tacta_status tacta_plan_matvec(tacta_plan plan, int32_t transpose, const double* x, double* y,
                               const tacta_options* opt) {
    set_error("");
    if (!plan || !plan->p || !x || !y) { set_error("NULL argument"); return TACTA_ERR_INVALID; }
    Plan* p = plan->p;
    Opts O = resolve(opt);
    CUDA_TRY(cudaSetDevice(p->device));
    const DevOperand& A = transpose ? p->At : p->A;
    const int64_t in_len = A.cols(), out_len = A.rows();
    // the input goes through a padded plan buffer: the staged kernels read 16-byte-rounded windows
    double* xin = transpose ? p->tmp_m : p->tmp_n;
    double* yout = transpose ? p->tmp_n : p->tmp_m;
    CUDA_TRY(cudaMemcpyAsync(xin, x, sizeof(double) * in_len, cudaMemcpyDefault, O.s));
    int64_t launches = 0;
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, &launches};
    CUDA_TRY(launch_spmv(L, A, xin, yout, EPI_NONE, EpiArgs{nullptr, nullptr, nullptr},
                         FinArgs{FIN_NONE, 0, nullptr}, GATE_FORCE));
    CUDA_TRY(cudaMemcpyAsync(y, yout, sizeof(double) * out_len, cudaMemcpyDefault, O.s));
    CUDA_TRY(cudaStreamSynchronize(O.s));
    return TACTA_OK;
}

tacta_status tacta_plan_residual(tacta_plan plan, int32_t transpose, const double* x, const double* b, double* r,
                                 const tacta_options* opt) {
    set_error("");
    if (!plan || !plan->p || !x || !b || !r) { set_error("NULL argument"); return TACTA_ERR_INVALID; }
    Plan* p = plan->p;
    Opts O = resolve(opt);
    CUDA_TRY(cudaSetDevice(p->device));
    const DevOperand& A = transpose ? p->At : p->A;
    const int64_t in_len = A.cols(), out_len = A.rows();
    // x through a padded plan buffer (the staged kernels read 16-byte-rounded windows), b
    // through another (max(m, n) long)
    double* xin = transpose ? p->tmp_m : p->tmp_n;
    double* yout = transpose ? p->tmp_n : p->tmp_m;
    CUDA_TRY(cudaMemcpyAsync(xin, x, sizeof(double) * in_len, cudaMemcpyDefault, O.s));
    CUDA_TRY(cudaMemcpyAsync(p->v, b, sizeof(double) * out_len, cudaMemcpyDefault, O.s));
    int64_t launches = 0;
    LaunchCtx L{O.s, p->ctl, p->partials, p->grid, &launches};
    CUDA_TRY(launch_spmv(L, A, xin, yout, EPI_RESID, EpiArgs{p->v, nullptr, nullptr},
                         FinArgs{FIN_NONE, 0, nullptr}, GATE_FORCE));
    CUDA_TRY(cudaMemcpyAsync(r, yout, sizeof(double) * out_len, cudaMemcpyDefault, O.s));
    CUDA_TRY(cudaStreamSynchronize(O.s));
    return TACTA_OK;
}

tacta_status tacta_plan_outer(tacta_plan plan, double alpha, const double* u, const double* v, double* out,
                              const tacta_options* opt) {
    set_error("");
    if (!plan || !plan->p || !u || !v || !out) { set_error("NULL argument"); return TACTA_ERR_INVALID; }
    Plan* p = plan->p;
    Opts O = resolve(opt);
    CUDA_TRY(cudaSetDevice(p->device));
    const int64_t len = p->A.nnz();
    // stage through plan buffers when the caller's arrays are on the host
    const double* du = u;
    const double* dv = v;
    double* dout = out;
    double* hold = nullptr;
    if (!p->on_device) {
        CUDA_TRY(cudaMemcpyAsync(p->tmp_m, u, sizeof(double) * p->m, cudaMemcpyHostToDevice, O.s));
        CUDA_TRY(cudaMemcpyAsync(p->tmp_n, v, sizeof(double) * p->n, cudaMemcpyHostToDevice, O.s));
        CUDA_TRY(cudaMalloc(&hold, sizeof(double) * std::max<int64_t>(len, 1)));
        CUDA_TRY(cudaMemcpyAsync(hold, out, sizeof(double) * len, cudaMemcpyHostToDevice, O.s));
        du = p->tmp_m;
        dv = p->tmp_n;
        dout = hold;
    }
    cudaError_t e = launch_outer_on_pattern(O.s, p->grid, p->A, alpha, du, dv, dout);
    if (e == cudaSuccess && hold) e = cudaMemcpyAsync(out, hold, sizeof(double) * len, cudaMemcpyDeviceToHost, O.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(O.s);
    if (hold) cudaFree(hold);
    CUDA_TRY(e);
    return TACTA_OK;
}

static tacta_status one_shot(int algo, const tacta_matrix* A, const double* b, const double* x0,
                             const tacta_options* opt, double* x_out, double* hist, int32_t hist_cap,
                             tacta_info* info) {
    tacta_plan plan = nullptr;
    tacta_status st = tacta_plan_create(A, opt, &plan);
    if (st != TACTA_OK) return st;
    st = plan_call(algo, plan, b, x0, opt, x_out, hist, hist_cap, info);
    std::string keep = get_error();
    tacta_plan_destroy(plan);
    set_error(keep);
    return st;
}

tacta_status cta_solve(const tacta_matrix* A, const double* b, const double* x0, const tacta_options* opt,
                       double* x_out, double* hist, int32_t hist_cap, tacta_info* info) {
    return one_shot(0, A, b, x0, opt, x_out, hist, hist_cap, info);
}
tacta_status ta_solve(const tacta_matrix* A, const double* b, const double* x0, const tacta_options* opt,
                      double* x_out, double* hist, int32_t hist_cap, tacta_info* info) {
    return one_shot(1, A, b, x0, opt, x_out, hist, hist_cap, info);
}
tacta_status ta_minnorm(const tacta_matrix* A, const double* b, const double* x0, const tacta_options* opt,
                        double* x_out, double* hist, int32_t hist_cap, tacta_info* info) {
    return one_shot(2, A, b, x0, opt, x_out, hist, hist_cap, info);
}

}  // extern "C"

extern "C" int32_t tacta_dia_tile_plan(int64_t rows, int64_t cols, int32_t k, const int32_t* offsets, int32_t tile,
                                       int32_t* runs, int32_t* sbase) {
    using namespace tacta;
    if (!offsets || !runs || !sbase || k < 1 || k > kDiaMax || rows < 1 || cols < 1 || tile < 0 ||
        (int64_t)tile * kTileRows >= rows)
        return -1;
    DiaOffsets d{};
    d.k = k;
    for (int i = 0; i < k; ++i) {
        d.off[i] = offsets[i];
        if (i > 0 && offsets[i] <= offsets[i - 1]) return -1;   // strictly ascending
    }
    int2 rr[kRunMax];
    int32_t sb[8];
    if (!dia_tile_plan(rows, cols, d, tile, rr, sb)) return 0;
    for (int i = 0; i < kRunMax; ++i) {
        runs[2 * i] = rr[i].x;
        runs[2 * i + 1] = rr[i].y;
    }
    for (int i = 0; i < 8; ++i) sbase[i] = sb[i];
    return 1;
}

extern "C" tacta_status tacta_column_partition(int64_t m, int64_t n, int64_t nnz, const int32_t* rowptr,
                                               const int32_t* colidx, int32_t nparts, int64_t* col_begin,
                                               int64_t* shard_nnz) {
    using namespace tacta;
    set_error("");
    if (!rowptr || (nnz > 0 && !colidx) || !col_begin || !shard_nnz) {
        set_error("NULL argument");
        return TACTA_ERR_INVALID;
    }
    if (m < 1 || n < 1 || nnz < 0 || nparts < 1 || nparts > n || rowptr[0] != 0 || rowptr[m] != nnz) {
        set_error("tacta_column_partition: need m, n >= 1, 1 <= nparts <= n, rowptr[0] = 0, rowptr[m] = nnz");
        return TACTA_ERR_INVALID;
    }
    // stored entries per column, then the prefix count of entries in columns < j
    std::vector<int64_t> before((size_t)n + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) {
        const int32_t c = colidx[k];
        if (c < 0 || c >= n) {
            set_error("tacta_column_partition: column index out of range");
            return TACTA_ERR_INVALID;
        }
        ++before[(size_t)c + 1];
    }
    for (int64_t j = 0; j < n; ++j) before[(size_t)j + 1] += before[(size_t)j];
    // shard g starts at the first column whose preceding entries reach g * nnz / nparts, and
    // every shard keeps at least one column
    col_begin[0] = 0;
    for (int32_t g = 1; g < nparts; ++g) {
        const int64_t want = (int64_t)((double)nnz * g / nparts);
        int64_t j = std::lower_bound(before.begin(), before.end(), want) - before.begin();
        j = std::max<int64_t>(j, col_begin[g - 1] + 1);
        j = std::min<int64_t>(j, n - (nparts - g));
        col_begin[g] = j;
    }
    col_begin[nparts] = n;
    for (int32_t g = 0; g < nparts; ++g) shard_nnz[g] = before[(size_t)col_begin[g + 1]] - before[(size_t)col_begin[g]];
    return TACTA_OK;
}

extern "C" int32_t tacta_aux_solve(const double* phi, int32_t t, double pivot_tol, double* alpha) {
    if (!phi || !alpha || t < 1 || t > kTMax) return -1;
    return hankel_solve_dev(phi, t, pivot_tol, alpha);
}
