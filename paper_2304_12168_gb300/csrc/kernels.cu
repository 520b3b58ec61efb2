// Device kernels of the TA / CTA hot path (sm_103a, FP64).
//
// Every per-iteration step of the paper's algorithms is one of:
//   * a matrix-vector product y = A x or y = Aᵀ r (Aᵀ is stored as its own
//     row-major operand), with a fused per-row epilogue and fused reductions
//     (norms for the moments phi_i of Eq. eqcoeff, the residual, the TA dots
//     of Eqs. vr / alph);
//   * a fused vector update (Eqs. CTAGEN7 / CTAGEN7A for CTA, the b'' / x''
//     update of Alg. 2.2 for TA) with the norms the next stop test needs;
//   * single-thread "finisher" code run by the last block of a reducing kernel:
//     the stop tests of Alg. 1.1 / 2.1 / 2.2, the t x t auxiliary (Hankel)
//     solve, the TA pivot test (Eq. eqlem2), step size (Eq. alph) and rho
//     growth.
//
// Reductions are deterministic: each block reduces its threads in a fixed
// shuffle tree, writes one partial per block, and the last block to finish
// (ticket from an atomic counter, no spinning) sums the partials in index
// order. No kernel waits on another block.
//
// GB300 notes: FP64 FMA issues at ~2 per SM-clock on this part, so each kernel
// spends exactly one FP64 FMA per stored nonzero (thread-per-row FMA chains,
// or warp-per-row chains for long rows) and keeps all index arithmetic in the
// integer pipes.
#include <algorithm>
#include <cfloat>
#include <cstdio>

#include "internal.h"
#include "hankel.cuh"
#include "mbarrier.cuh"
#include "rowtiles.cuh"
#include "finish.cuh"
#include "aux_step.cuh"

namespace tacta {

template <int EPI>
struct EpiRed {
    static constexpr int value = (EPI == EPI_RESID || EPI == EPI_TAPIVOT || EPI == EPI_RESID_F32) ? 2 : 1;
};

// ------------------------------------------------------------------ operand access

struct CsrAcc {
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ colidx;
    const double* __restrict__ vals;
    int64_t rows;
    __device__ __forceinline__ int64_t begin(int64_t r) const { return __ldg(rowptr + r); }
    __device__ __forceinline__ int64_t end(int64_t r) const { return __ldg(rowptr + r + 1); }
    __device__ __forceinline__ int64_t col(int64_t k, int64_t) const { return __ldg(colidx + k); }
    __device__ __forceinline__ double val(int64_t k) const { return __ldg(vals + k); }
};

template <int EPI>
__device__ __forceinline__ void epilogue(int64_t row, double sum, double* __restrict__ y,
                                         const EpiArgs& e, double s, double& a0, double& a1) {
    if (EPI == EPI_NONE) {
        y[row] = sum;
    } else if (EPI == EPI_NORM) {
        y[row] = sum;
        a0 = fma(sum, sum, a0);
    } else if (EPI == EPI_NORM_POS) {
        const double v = sum > 0.0 ? sum : 0.0;
        y[row] = v;
        a0 = fma(v, v, a0);
    } else if (EPI == EPI_RESID) {
        const double bv = __ldg(e.b + row);
        const double v = bv - sum;
        y[row] = v;
        a0 = fma(v, v, a0);
        a1 = fma(v, bv, a1);
    } else if (EPI == EPI_TAPIVOT) {  // v = s (A c); w = v - b' = v - b + d, stored for the update
        const double v = s * sum;
        const double dv = __ldg(e.d + row);
        const double w = (v - __ldg(e.b + row)) + dv;
        y[row] = w;
        a0 = fma(dv, w, a0);
        a1 = fma(w, w, a1);
    } else {  // EPI_RESID_F32: FP64 residual, stored in FP32 for the mixed-precision chain
        const double bv = __ldg(e.b + row);
        const double v = bv - sum;
        e.yf[row] = (float)v;
        a0 = fma(v, v, a0);
        a1 = fma(v, bv, a1);
    }
}

// Thread per row: one FMA chain per row (short rows).
template <class Acc, int EPI>
__global__ void __launch_bounds__(kBlock)
spmv_scalar(Acc A, const double* __restrict__ x, double* __restrict__ y, EpiArgs e, Ctl* ctl,
            double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    const double s = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
    double a0 = 0.0, a1 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the loop runs while any lane of the warp has a row, so shuffles stay converged
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < A.rows; base += stride) {
        const int64_t row = base + threadIdx.x;
        const bool active = row < A.rows;
        const int64_t b = active ? A.begin(row) : 0, en = active ? A.end(row) : 0;
        const int len = (int)(en - b);
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        double sum = 0.0;
        for (int u = 0; u < maxlen; ++u)
            if (u < len) sum = fma(A.val(b + u), __ldg(x + A.col(b + u, b)), sum);
        if (active) epilogue<EPI>(row, sum, y, e, s, a0, a1);
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<EpiRed<EPI>::value>(a0, a1, ctl, partials, f);
}

// Warp per row: lanes stride over the row, shuffle-sum at the end (long rows).
template <class Acc, int EPI>
__global__ void __launch_bounds__(kBlock)
spmv_warp(Acc A, const double* __restrict__ x, double* __restrict__ y, EpiArgs e, Ctl* ctl,
          double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    const double s = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
    double a0 = 0.0, a1 = 0.0;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < A.rows;
         row += warps) {
        const int64_t b = A.begin(row), en = A.end(row);
        double sum = 0.0;
        for (int64_t k = b + lane; k < en; k += 32) sum = fma(A.val(k), __ldg(x + A.col(k, b)), sum);
        sum = warp_sum(sum);
        if (lane == 0) epilogue<EPI>(row, sum, y, e, s, a0, a1);
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<EpiRed<EPI>::value>(a0, a1, ctl, partials, f);
}

// ------------------------------------------------------------------ TMA-staged row tiles
//
// A tile is up to kTileRows consecutive rows holding at most CAP nonzeros. One
// elected thread copies the tile's values, column indices and row offsets into
// shared memory with cp.async.bulk (1-D TMA), completion tracked by an
// mbarrier; two stages, so tile j+1 streams in while tile j is multiplied.
// Every thread then runs the FMA chain of its own row out of shared memory,
// gathering x through the read-only path. Bulk copies start on 16-byte
// boundaries: each window is rounded outwards and the padded CSR arrays
// (kPad*) keep the rounded end inside the allocation.

template <int CAP>
struct __align__(16) TileStage {
    double vals[CAP + 2];
    int32_t cols[CAP + 4];
    int32_t rp[kTileRows + 8];
};

size_t spmv_tiled_smem(int cap) {
    return cap <= kTileCapSmall ? 2 * sizeof(TileStage<kTileCapSmall>) : 2 * sizeof(TileStage<kTileCapLarge>);
}

// issue the bulk copies of tile d into stage st (one thread)
template <int CAP>
__device__ __forceinline__ void tile_issue(const int4 d, TileStage<CAP>* st, uint64_t* bar,
                                           const int32_t* rowptr, const int32_t* colidx,
                                           const double* vals) {
    const int a0 = d.z & ~1, c0 = d.z & ~3, r0 = d.x & ~3;
    const uint32_t bv = d.w > d.z ? round16((uint32_t)(d.w - a0) * 8u) : 0u;
    const uint32_t bc = d.w > d.z ? round16((uint32_t)(d.w - c0) * 4u) : 0u;
    const uint32_t br = round16((uint32_t)(d.y + 1 - r0) * 4u);
    mbar_expect_tx(bar, bv + bc + br);
    if (bv) bulk_g2s(st->vals, vals + a0, bv, bar);
    if (bc) bulk_g2s(st->cols, colidx + c0, bc, bar);
    bulk_g2s(st->rp, rowptr + r0, br, bar);
}

// Registers a thread carries for one row of a tile: the row's first entries of x
// (gathered ahead of use) and where the row's values sit in its stage.
constexpr int kAhead = 6;
struct RowRegs {
    double xv[kAhead];
    int kb;        // first value of the row, relative to the stage's value window
    int cb;        // same for the column window
    int len;
    int maxlen;    // max len over the warp (warp-uniform FMA trip count)
    bool active;
};

template <int CAP>
__device__ __forceinline__ void row_fetch(const TileStage<CAP>* S, const int4 d, int tid, bool ok,
                                          const double* __restrict__ x, RowRegs& R) {
    const int row = d.x + tid;
    R.active = ok && row < d.y;
    R.len = 0;
    R.kb = 0;
    R.cb = 0;
    if (R.active) {
        const int r0 = d.x & ~3;
        const int k0 = S->rp[row - r0];
        R.len = S->rp[row + 1 - r0] - k0;
        R.kb = k0 - (d.z & ~1);
        R.cb = k0 - (d.z & ~3);
    }
    R.maxlen = __reduce_max_sync(0xffffffffu, R.len);
#pragma unroll
    for (int u = 0; u < kAhead; ++u)
        if (u < R.len) R.xv[u] = __ldg(x + S->cols[R.cb + u]);
}

template <int CAP>
__device__ __forceinline__ double row_dot(const TileStage<CAP>* S, const RowRegs& R,
                                          const double* __restrict__ x) {
    // a predicated-off FP64 FMA still costs a full warp slot on GB300: the trip
    // count is the warp-uniform maximum row length
    double sum = 0.0;
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
        if (u >= R.maxlen) break;
        if (u < R.len) sum = fma(S->vals[R.kb + u], R.xv[u], sum);
    }
    for (int u = kAhead; u < R.maxlen; ++u)
        if (u < R.len) sum = fma(S->vals[R.kb + u], __ldg(x + S->cols[R.cb + u]), sum);
    return sum;
}

template <int CAP, int EPI>
__global__ void __launch_bounds__(kTileRows)
spmv_tiled(const int4* __restrict__ tiles, int ntiles, const int32_t* __restrict__ rowptr,
           const int32_t* __restrict__ colidx, const double* __restrict__ vals,
           const double* __restrict__ x, double* __restrict__ y, EpiArgs e, Ctl* ctl, double* partials,
           FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileStage<CAP>* st = reinterpret_cast<TileStage<CAP>*>(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int failed;
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        for (int j = 0; j < 2; ++j) {
            const int t = blockIdx.x + j * G;
            if (t < ntiles) tile_issue<CAP>(__ldg(tiles + t), st + j, bar + j, rowptr, colidx, vals);
        }
    }
    __syncthreads();
    const double s = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
    double a0 = 0.0, a1 = 0.0;
    // Software pipeline over this block's tiles j = 0, 1, ...: tile j+1's x values
    // are gathered (loads in flight) before tile j's FMA chains run on the values
    // gathered one step earlier; tile j+2's bulk copy is issued once every thread
    // is done with tile j's stage.
    RowRegs cur;
    int4 dcur = make_int4(0, 0, 0, 0);
    if (blockIdx.x < ntiles) {
        dcur = __ldg(tiles + blockIdx.x);
        bool ok = mbar_wait_bounded(bar + 0, 0u);
        if (!ok) { failed = 1; atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT); }
        row_fetch<CAP>(st + 0, dcur, tid, ok, x, cur);
    }
    for (int j = 0;; ++j) {
        const int t = blockIdx.x + j * G;
        if (t >= ntiles) break;
        const int sidx = j & 1;
        RowRegs nxt;
        int4 dnxt = make_int4(0, 0, 0, 0);
        const int tn = t + G;
        if (tn < ntiles) {
            dnxt = __ldg(tiles + tn);
            bool ok = !failed && mbar_wait_bounded(bar + (sidx ^ 1), (uint32_t)(((j + 1) >> 1) & 1));
            if (!ok) { failed = 1; atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT); }
            row_fetch<CAP>(st + (sidx ^ 1), dnxt, tid, ok, x, nxt);
        }
        const double sum = row_dot<CAP>(st + sidx, cur, x);
        if (cur.active) epilogue<EPI>(dcur.x + tid, sum, y, e, s, a0, a1);
        __syncthreads();   // stage sidx is free again
        if (tid == 0 && !failed) {
            const int t2 = t + 2 * G;
            if (t2 < ntiles) tile_issue<CAP>(__ldg(tiles + t2), st + sidx, bar + sidx, rowptr, colidx, vals);
        }
        cur = nxt;
        dcur = dnxt;
    }
    if (failed && tid == 0) {
        // give the copies still in flight a bounded chance to land before the block exits
        for (int j = 0; j < 2; ++j) mbar_wait_bounded(bar + j, 0u);
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<EpiRed<EPI>::value>(a0, a1, ctl, partials, f);
}

// ------------------------------------------------------------------ banded variant: x window staged too
//
// When every tile's columns fall in a window of at most kXSpan entries of x
// (banded operands such as stencils), the bulk copies also bring that window
// of x into shared memory, so each row's FMA chain reads values, indices and
// x from shared memory and the narrow FP64 pipe is not left waiting on global
// gathers.

template <int CAP, int XS>
struct __align__(16) TileStageX {
    double vals[CAP + 2];
    int32_t cols[CAP + 4];
    int32_t rp[kTileRows + 8];
    double xs[XS + 2];
};

// two instances: a compact one (three blocks per SM) for tiles of <= 1280 nonzeros whose
// x windows span <= 2304 entries (e.g. 5-point stencils up to 1000 columns of bandwidth),
// and the general one (two blocks per SM)
constexpr int kXCapCompact = kXCapCompactPlan, kXSpanCompact = kXSpanCompactPlan;

template <int CAP, int XS>
size_t spmv_tiled_x_smem() { return 2 * sizeof(TileStageX<CAP, XS>); }

template <int CAP, int XS>
__device__ __forceinline__ void tile_issue_x(const int4 d, const int2 w, TileStageX<CAP, XS>* st,
                                             uint64_t* bar, const int32_t* rowptr,
                                             const int32_t* colidx, const double* vals,
                                             const double* x) {
    const int a0 = d.z & ~1, c0 = d.z & ~3, r0 = d.x & ~3, x0 = w.x & ~1;
    const uint32_t bv = d.w > d.z ? round16((uint32_t)(d.w - a0) * 8u) : 0u;
    const uint32_t bc = d.w > d.z ? round16((uint32_t)(d.w - c0) * 4u) : 0u;
    const uint32_t br = round16((uint32_t)(d.y + 1 - r0) * 4u);
    const uint32_t bx = d.w > d.z ? round16((uint32_t)(w.y + 1 - x0) * 8u) : 0u;
    mbar_expect_tx(bar, bv + bc + br + bx);
    if (bv) bulk_g2s(st->vals, vals + a0, bv, bar);
    if (bc) bulk_g2s(st->cols, colidx + c0, bc, bar);
    bulk_g2s(st->rp, rowptr + r0, br, bar);
    if (bx) bulk_g2s(st->xs, x + x0, bx, bar);
}

template <int CAP, int XS, int EPI>
__global__ void __launch_bounds__(kTileRows)
spmv_tiled_x(const int4* __restrict__ tiles, const int2* __restrict__ xwin, int ntiles,
             const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
             const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
             EpiArgs e, Ctl* ctl, double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileStageX<CAP, XS>* st = reinterpret_cast<TileStageX<CAP, XS>*>(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int failed;
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        for (int j = 0; j < 2; ++j) {
            const int t = blockIdx.x + j * G;
            if (t < ntiles)
                tile_issue_x<CAP, XS>(__ldg(tiles + t), __ldg(xwin + t), st + j, bar + j, rowptr, colidx, vals, x);
        }
    }
    __syncthreads();
    const double s = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
    double a0 = 0.0, a1 = 0.0;
    for (int j = 0;; ++j) {
        const int t = blockIdx.x + j * G;
        if (t >= ntiles) break;
        const int sidx = j & 1;
        const int4 d = __ldg(tiles + t);
        const int xw0 = __ldg(&xwin[t].x) & ~1;
        const bool ok = !failed && mbar_wait_bounded(bar + sidx, (uint32_t)((j >> 1) & 1));
        if (!ok) {
            failed = 1;
            atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
        }
        const TileStageX<CAP, XS>* S = st + sidx;
        const int row = d.x + tid;
        const bool active = ok && row < d.y;
        int kb = 0, len = 0;
        if (active) {
            const int r0 = d.x & ~3;
            kb = S->rp[row - r0];
            len = S->rp[row + 1 - r0] - kb;
        }
        // trip count = warp-uniform max row length (a masked FP64 FMA costs a full slot)
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        const int vb = kb - (d.z & ~1), cb = kb - (d.z & ~3);
        double sum = 0.0;
        for (int u = 0; u < maxlen; ++u)
            if (u < len) sum = fma(S->vals[vb + u], S->xs[S->cols[cb + u] - xw0], sum);
        if (active) epilogue<EPI>(row, sum, y, e, s, a0, a1);
        __syncthreads();   // stage sidx is free again
        if (tid == 0 && !failed) {
            const int t2 = t + 2 * G;
            if (t2 < ntiles)
                tile_issue_x<CAP, XS>(__ldg(tiles + t2), __ldg(xwin + t2), st + sidx, bar + sidx, rowptr,
                                      colidx, vals, x);
        }
    }
    if (failed && tid == 0) {
        for (int j = 0; j < 2; ++j) mbar_wait_bounded(bar + j, 0u);
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<EpiRed<EPI>::value>(a0, a1, ctl, partials, f);
}

template <int EPI>
static cudaError_t spmv_tiled_x_launch(const LaunchCtx& L, const DevCSR& A, const double* x, double* y,
                                       EpiArgs e, FinArgs f, int gate) {
    const int sms = L.max_grid / 8;
    if (A.cap == kXCapCompact) {   // two 36 KB stages per block: three blocks per SM
        const int grid = std::min(A.ntiles, std::max(1, sms * 3));
        spmv_tiled_x<kXCapCompact, kXSpanCompact, EPI>
            <<<grid, kTileRows, spmv_tiled_x_smem<kXCapCompact, kXSpanCompact>(), L.stream>>>(
                A.tiles, A.xwin, A.ntiles, A.rowptr, A.colidx, A.vals, x, y, e, L.ctl, L.partials, f, gate);
    } else {                       // two 46 KB stages per block: two blocks per SM
        const int grid = std::min(A.ntiles, std::max(1, sms * 2));
        spmv_tiled_x<kTileCapSmall, kXSpan, EPI>
            <<<grid, kTileRows, spmv_tiled_x_smem<kTileCapSmall, kXSpan>(), L.stream>>>(
                A.tiles, A.xwin, A.ntiles, A.rowptr, A.colidx, A.vals, x, y, e, L.ctl, L.partials, f, gate);
    }
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ run-staged, warp-specialised
//
// Run-staged tiles without a block-wide barrier per tile: one producer warp
// streams tiles into a ring of S stages (a "full"
// mbarrier per stage completes when the tile's bytes land), and each of the eight
// consumer warps multiplies its own 32 rows of a tile as soon as it has landed,
// then arrives on the stage's "empty" mbarrier; the producer refills a stage once
// all eight warps have released it. Warps drift apart instead of waiting for the
// slowest one, which spreads shared-memory and FP64 issue over time.



template <int S> constexpr int rw_blocks_per_sm() { return S == 2 ? 4 : 3; }

template <int S, int EPI>
__global__ void __launch_bounds__(kRwThreads, rw_blocks_per_sm<S>())
spmv_tiled_rw(const int4* __restrict__ tiles, const int2* __restrict__ runs, int ntiles,
              const int32_t* __restrict__ rowptr, const uint16_t* __restrict__ lcol,
              const double* __restrict__ vals, const double* __restrict__ x, double* __restrict__ y,
              EpiArgs e, Ctl* ctl, double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileStageR* st = reinterpret_cast<TileStageR*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ volatile int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRwConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    __syncthreads();
    double a0 = 0.0, a1 = 0.0;
    int last_use[S];   // producer lane: the last use issued into each stage
    for (int k = 0; k < S; ++k) last_use[k] = -1;
    if (warp == kRwConsumers) {
        // producer: lane 0 issues tile j into stage j % S once its previous use is released;
        // the warp's lanes prefetch the tiles' metadata
        TilePrefetch pf;
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles || __any_sync(0xffffffffu, failed != 0)) break;   // one decision per warp
            const TileMeta tm = pf.get(j, tiles, runs, ntiles, G, lane);
            if (lane == 0) {
                const int k = j % S, u = j / S;
                if (u > 0 && !mbar_wait_bounded(&empty[k], (uint32_t)((u - 1) & 1))) {
                    failed = 1;
                    atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                } else {
                    st[k].desc = tm.d;   // visible to the consumers through the stage's mbarrier
                    tile_issue_r(tm, st + k, &full[k], rowptr, lcol, vals, x);
                    last_use[k] = u;
                }
            }
            __syncwarp();
        }
    } else {
        const double s = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles) break;
            const int k = j % S;
            const bool ok = !failed && mbar_wait_bounded(&full[k], (uint32_t)((j / S) & 1));
            if (!__all_sync(0xffffffffu, ok)) {   // the warp takes one path
                if (lane == 0) {
                    failed = 1;
                    atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                }
                break;
            }
            int row;
            bool active;
            const double sum = rw_row_dot(st + k, warp, lane, row, active);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[k]);   // this warp is done with stage k
            if (active) epilogue<EPI>(row, sum, y, e, s, a0, a1);
        }
    }
    __syncthreads();
    if (failed && warp == kRwConsumers && lane == 0) {
        // a wait gave up: let every copy already issued land before the block exits
        for (int k = 0; k < S; ++k)
            if (last_use[k] >= 0) mbar_wait_bounded(&full[k], (uint32_t)(last_use[k] & 1));
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE)
        reduce_and_finish<EpiRed<EPI>::value, kRwThreads>(a0, a1, ctl, partials, f);
}

template <int S>
size_t spmv_tiled_rw_smem() { return (size_t)S * sizeof(TileStageR); }

// The same warp-specialised product on the diagonal form (operands whose nonzeros lie on
// at most kDiaMax diagonals): only the values move, and every row runs its FMAs in
// ascending column order, so the results are those of spmv_tiled_rw whenever the CSR rows
// list their columns in ascending order.
template <int S, int EPI>
__global__ void __launch_bounds__(kRwThreads, rw_blocks_per_sm<S>())
spmv_dia(ChainOpsDia<double> ops, const double* __restrict__ x, double* __restrict__ y, EpiArgs e, Ctl* ctl,
         double* partials, FinArgs f, int gate) {
    using F = DiaFmt<double>;
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    F::Stage* st = reinterpret_cast<F::Stage*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ volatile int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, ntiles = ops.ntiles[0];
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRwConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    __syncthreads();
    double a0 = 0.0, a1 = 0.0;
    int last_use[S];
    for (int k = 0; k < S; ++k) last_use[k] = -1;
    if (warp == kRwConsumers) {
        F::Prefetch pf;
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles || __any_sync(0xffffffffu, failed != 0)) break;   // one decision per warp
            const F::Meta tm = pf.get(j, ops, 0, G, lane);
            if (lane == 0) {
                const int k = j % S, u = j / S;
                if (u > 0 && !mbar_wait_bounded(&empty[k], (uint32_t)((u - 1) & 1))) {
                    failed = 1;
                    atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                } else {
                    F::issue_mat(tm, st + k, &full[k], ops, 0);
                    F::issue_x(tm, st + k, &full[k], x);
                    last_use[k] = u;
                }
            }
            __syncwarp();
        }
    } else {
        const double s = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles) break;
            const int k = j % S;
            const bool ok = !failed && mbar_wait_bounded(&full[k], (uint32_t)((j / S) & 1));
            if (!__all_sync(0xffffffffu, ok)) {   // the warp takes one path
                if (lane == 0) {
                    failed = 1;
                    atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                }
                break;
            }
            int row;
            bool active;
            const double sum = F::row_dot(st + k, ops, warp, lane, row, active);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[k]);
            if (active) epilogue<EPI>(row, sum, y, e, s, a0, a1);
        }
    }
    __syncthreads();
    if (failed && warp == kRwConsumers && lane == 0) {
        for (int k = 0; k < S; ++k)
            if (last_use[k] >= 0) mbar_wait_bounded(&full[k], (uint32_t)(last_use[k] & 1));
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE)
        reduce_and_finish<EpiRed<EPI>::value, kRwThreads>(a0, a1, ctl, partials, f);
}

template <int S, int EPI>
static cudaError_t spmv_dia_launch(const LaunchCtx& L, const DevCSR& A, const double* x, double* y, EpiArgs e,
                                   FinArgs f, int gate) {
    static const char attr_key = 0;
    const size_t smem = (size_t)S * sizeof(DiaFmt<double>::Stage);
    if (!done_on_device(&attr_key)) {
        const cudaError_t e2 = cudaFuncSetAttribute(spmv_dia<S, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem);
        if (e2 != cudaSuccess) return e2;
        mark_done_on_device(&attr_key);
    }
    ChainOpsDia<double> ops{};
    ops.vals[0] = A.dia.vals;
    ops.mask[0] = A.dia.mask;
    ops.runs[0] = A.dia.runs;
    ops.sbase[0] = A.dia.sbase;
    ops.ntiles[0] = A.dia.ntiles;
    ops.rows[0] = (int)A.rows;
    ops.k = A.dia.k;
    const int sms = L.max_grid / 8;
    const int grid = std::min(A.dia.ntiles, std::max(1, sms * rw_blocks_per_sm<S>()));
    spmv_dia<S, EPI><<<grid, kRwThreads, smem, L.stream>>>(ops, x, y, e, L.ctl, L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}


template <int S, int EPI>
static cudaError_t spmv_tiled_rw_launch(const LaunchCtx& L, const DevCSR& A, const double* x, double* y,
                                        EpiArgs e, FinArgs f, int gate) {
    const int sms = L.max_grid / 8;
    const int grid = std::min(A.ntiles, std::max(1, sms * rw_blocks_per_sm<S>()));
    spmv_tiled_rw<S, EPI><<<grid, kRwThreads, spmv_tiled_rw_smem<S>(), L.stream>>>(
        A.tiles, A.runs, A.ntiles, A.rowptr, A.lcol, A.vals, x, y, e, L.ctl, L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t spmv_tiled_prepare() {
    static const char done_key = 0;
    if (done_on_device(&done_key)) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define TACTA_TILED_ATTR(CAP, EPI)                                                                   \
    if (e == cudaSuccess)                                                                            \
        e = cudaFuncSetAttribute(spmv_tiled<CAP, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 (int)spmv_tiled_smem(CAP));
    TACTA_TILED_ATTR(kTileCapSmall, EPI_NONE) TACTA_TILED_ATTR(kTileCapSmall, EPI_NORM)
    TACTA_TILED_ATTR(kTileCapSmall, EPI_RESID) TACTA_TILED_ATTR(kTileCapSmall, EPI_TAPIVOT)
    TACTA_TILED_ATTR(kTileCapLarge, EPI_NONE) TACTA_TILED_ATTR(kTileCapLarge, EPI_NORM)
    TACTA_TILED_ATTR(kTileCapLarge, EPI_RESID) TACTA_TILED_ATTR(kTileCapLarge, EPI_TAPIVOT)
    TACTA_TILED_ATTR(kTileCapSmall, EPI_RESID_F32) TACTA_TILED_ATTR(kTileCapLarge, EPI_RESID_F32)
    TACTA_TILED_ATTR(kTileCapSmall, EPI_NORM_POS) TACTA_TILED_ATTR(kTileCapLarge, EPI_NORM_POS)
#undef TACTA_TILED_ATTR
#define TACTA_TILED_X_ATTR(EPI)                                                                          \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(spmv_tiled_x<kTileCapSmall, kXSpan, EPI>,                               \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                                 (int)spmv_tiled_x_smem<kTileCapSmall, kXSpan>());                       \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(spmv_tiled_x<kXCapCompact, kXSpanCompact, EPI>,                         \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                                 (int)spmv_tiled_x_smem<kXCapCompact, kXSpanCompact>());
    TACTA_TILED_X_ATTR(EPI_NONE) TACTA_TILED_X_ATTR(EPI_NORM) TACTA_TILED_X_ATTR(EPI_RESID)
    TACTA_TILED_X_ATTR(EPI_TAPIVOT) TACTA_TILED_X_ATTR(EPI_RESID_F32) TACTA_TILED_X_ATTR(EPI_NORM_POS)

#define TACTA_TILED_RW_ATTR(EPI)                                                                         \
    if (e == cudaSuccess)                                                                                \
        e = cudaFuncSetAttribute(spmv_tiled_rw<kRwStages, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)spmv_tiled_rw_smem<kRwStages>());
    TACTA_TILED_RW_ATTR(EPI_NONE) TACTA_TILED_RW_ATTR(EPI_NORM) TACTA_TILED_RW_ATTR(EPI_RESID)
    TACTA_TILED_RW_ATTR(EPI_TAPIVOT) TACTA_TILED_RW_ATTR(EPI_RESID_F32) TACTA_TILED_RW_ATTR(EPI_NORM_POS)
#undef TACTA_TILED_RW_ATTR

#undef TACTA_TILED_X_ATTR
    if (e == cudaSuccess) mark_done_on_device(&done_key);
    return e;
}

template <int EPI>
static cudaError_t spmv_tiled_launch(const LaunchCtx& L, const DevCSR& A, const double* x, double* y,
                                     EpiArgs e, FinArgs f, int gate) {
    const int per_sm = A.cap <= kTileCapSmall ? 4 : 1;
    int grid = std::min(A.ntiles, std::max(1, (L.max_grid / 8) * per_sm));
    if (grid < 1) grid = 1;
    const size_t sm = spmv_tiled_smem(A.cap);
    if (A.cap <= kTileCapSmall)
        spmv_tiled<kTileCapSmall, EPI><<<grid, kTileRows, sm, L.stream>>>(
            A.tiles, A.ntiles, A.rowptr, A.colidx, A.vals, x, y, e, L.ctl, L.partials, f, gate);
    else
        spmv_tiled<kTileCapLarge, EPI><<<grid, kTileRows, sm, L.stream>>>(
            A.tiles, A.ntiles, A.rowptr, A.colidx, A.vals, x, y, e, L.ctl, L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

template <class Acc, int EPI>
static cudaError_t spmv_dispatch_epi(const LaunchCtx& L, int kind, const Acc& acc, const double* x,
                                     double* y, EpiArgs e, FinArgs f, int gate) {
    const int grid = L.max_grid;
    if (kind == 0)
        spmv_scalar<Acc, EPI><<<grid, kBlock, 0, L.stream>>>(acc, x, y, e, L.ctl, L.partials, f, gate);
    else
        spmv_warp<Acc, EPI><<<grid, kBlock, 0, L.stream>>>(acc, x, y, e, L.ctl, L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

// Dense FP64 product, every epilogue: row-major A, WPR warps share a row (enough warps in
// flight for HBM and the FP64 pipe when rows are few and long), each summing an
// interleaved share of the row's 16-byte vectors with four independent FMA chains; the
// WPR partial sums meet in shared memory in warp order (deterministic), and one lane runs
// the row's epilogue.
template <int WPR, int EPI>
__global__ void __launch_bounds__(kBlock)
dense_rows(int64_t rows, int64_t cols, const double* __restrict__ A, const double* __restrict__ x,
           double* __restrict__ y, EpiArgs e, Ctl* ctl, double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    const double sv = (EPI == EPI_TAPIVOT) ? ctl->s : 0.0;
    constexpr int RPB = (kBlock / 32) / WPR;   // rows per block and pass
    __shared__ double red[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rl = warp / WPR, part = warp % WPR;
    const bool vec = (cols & 1) == 0;          // rows start 16-byte aligned
    double a0 = 0.0, a1 = 0.0;
    const int64_t groups = (rows + RPB - 1) / RPB;
    for (int64_t gidx = blockIdx.x; gidx < groups; gidx += gridDim.x) {
        const int64_t row = gidx * RPB + rl;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        if (row < rows) {
            const double* a = A + row * cols;
            if (vec) {
                const double2* a2 = reinterpret_cast<const double2*>(a);
                const double2* x2 = reinterpret_cast<const double2*>(x);
                const int64_t nv = cols >> 1, step = 32 * WPR;
                int64_t c = part * 32 + lane;
                for (; c + step < nv; c += 2 * step) {
                    const double2 p0 = __ldg(a2 + c), p1 = __ldg(a2 + c + step);
                    const double2 q0 = __ldg(x2 + c), q1 = __ldg(x2 + c + step);
                    s0 = fma(p0.x, q0.x, s0);
                    s1 = fma(p0.y, q0.y, s1);
                    s2 = fma(p1.x, q1.x, s2);
                    s3 = fma(p1.y, q1.y, s3);
                }
                if (c < nv) {
                    const double2 p0 = __ldg(a2 + c), q0 = __ldg(x2 + c);
                    s0 = fma(p0.x, q0.x, s0);
                    s1 = fma(p0.y, q0.y, s1);
                }
            } else {
                for (int64_t c = part * 32 + lane; c < cols; c += 32 * WPR) s0 = fma(__ldg(a + c), __ldg(x + c), s0);
            }
        }
        double sum = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (WPR == 1) {
            if (lane == 0 && row < rows) epilogue<EPI>(row, sum, y, e, sv, a0, a1);
        } else {
            if (lane == 0) red[warp] = sum;
            __syncthreads();
            if (part == 0 && lane == 0 && row < rows) {
                double t = red[warp];
                for (int q = 1; q < WPR; ++q) t += red[warp + q];
                epilogue<EPI>(row, t, y, e, sv, a0, a1);
            }
            __syncthreads();
        }
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<EpiRed<EPI>::value>(a0, a1, ctl, partials, f);
}

// Warps per row of the dense products: rows are split among warps until the launch has
// about as many warps as the grid holds (rows few and long), keeping at least 256 columns
// per warp; the grid is at most max_grid blocks (the partials buffer), one group of
// 8 / wpr rows per block and pass.
static int dense_wpr(const LaunchCtx& L, int64_t rows, int64_t cols) {
    const int64_t want = (int64_t)L.max_grid * (kBlock / 32);
    int wpr = 1;
    while (wpr < 8 && rows * wpr * 2 <= want && cols >= 256LL * wpr) wpr *= 2;
    return wpr;
}

static int dense_grid(const LaunchCtx& L, int64_t rows, int wpr) {
    const int64_t rpb = (kBlock / 32) / wpr;
    const int64_t groups = (rows + rpb - 1) / rpb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)L.max_grid));
}

template <int EPI>
static cudaError_t dense_launch(const LaunchCtx& L, const DevDense& A, const double* x, double* y, EpiArgs e,
                                FinArgs f, int gate) {
    const int wpr = dense_wpr(L, A.rows, A.cols);
    const int grid = dense_grid(L, A.rows, wpr);
    if (L.launches) ++*L.launches;
    switch (wpr) {
    case 1: dense_rows<1, EPI><<<grid, kBlock, 0, L.stream>>>(A.rows, A.cols, A.vals, x, y, e, L.ctl, L.partials, f, gate); break;
    case 2: dense_rows<2, EPI><<<grid, kBlock, 0, L.stream>>>(A.rows, A.cols, A.vals, x, y, e, L.ctl, L.partials, f, gate); break;
    case 4: dense_rows<4, EPI><<<grid, kBlock, 0, L.stream>>>(A.rows, A.cols, A.vals, x, y, e, L.ctl, L.partials, f, gate); break;
    default: dense_rows<8, EPI><<<grid, kBlock, 0, L.stream>>>(A.rows, A.cols, A.vals, x, y, e, L.ctl, L.partials, f, gate); break;
    }
    return cudaGetLastError();
}

template <class Acc>
static cudaError_t spmv_dispatch(const LaunchCtx& L, int kind, const Acc& acc, const double* x,
                                 double* y, int epi, EpiArgs e, FinArgs f, int gate) {
    switch (epi) {
    case EPI_NONE: return spmv_dispatch_epi<Acc, EPI_NONE>(L, kind, acc, x, y, e, f, gate);
    case EPI_NORM: return spmv_dispatch_epi<Acc, EPI_NORM>(L, kind, acc, x, y, e, f, gate);
    case EPI_RESID: return spmv_dispatch_epi<Acc, EPI_RESID>(L, kind, acc, x, y, e, f, gate);
    case EPI_RESID_F32: return spmv_dispatch_epi<Acc, EPI_RESID_F32>(L, kind, acc, x, y, e, f, gate);
    case EPI_NORM_POS: return spmv_dispatch_epi<Acc, EPI_NORM_POS>(L, kind, acc, x, y, e, f, gate);
    default: return spmv_dispatch_epi<Acc, EPI_TAPIVOT>(L, kind, acc, x, y, e, f, gate);
    }
}

cudaError_t launch_spmv(const LaunchCtx& L, const DevOperand& A, const double* x, double* y,
                        int epi, EpiArgs e, FinArgs f, int gate) {
    if (A.format == TACTA_CSR && A.csr.dia.k > 0) {
        switch (epi) {
        case EPI_NONE: return spmv_dia_launch<kRwStages, EPI_NONE>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM: return spmv_dia_launch<kRwStages, EPI_NORM>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID: return spmv_dia_launch<kRwStages, EPI_RESID>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID_F32: return spmv_dia_launch<kRwStages, EPI_RESID_F32>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM_POS: return spmv_dia_launch<kRwStages, EPI_NORM_POS>(L, A.csr, x, y, e, f, gate);
        default: return spmv_dia_launch<kRwStages, EPI_TAPIVOT>(L, A.csr, x, y, e, f, gate);
        }
    }
    if (A.format == TACTA_CSR && A.csr.cfg.kind == 3 && A.csr.lcol) {
        switch (epi) {
        case EPI_NONE: return spmv_tiled_rw_launch<kRwStages, EPI_NONE>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM: return spmv_tiled_rw_launch<kRwStages, EPI_NORM>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID: return spmv_tiled_rw_launch<kRwStages, EPI_RESID>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID_F32: return spmv_tiled_rw_launch<kRwStages, EPI_RESID_F32>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM_POS: return spmv_tiled_rw_launch<kRwStages, EPI_NORM_POS>(L, A.csr, x, y, e, f, gate);
        default: return spmv_tiled_rw_launch<kRwStages, EPI_TAPIVOT>(L, A.csr, x, y, e, f, gate);
        }
    }
    if (A.format == TACTA_CSR && A.csr.cfg.kind == 3) {
        switch (epi) {
        case EPI_NONE: return spmv_tiled_x_launch<EPI_NONE>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM: return spmv_tiled_x_launch<EPI_NORM>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID: return spmv_tiled_x_launch<EPI_RESID>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID_F32: return spmv_tiled_x_launch<EPI_RESID_F32>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM_POS: return spmv_tiled_x_launch<EPI_NORM_POS>(L, A.csr, x, y, e, f, gate);
        default: return spmv_tiled_x_launch<EPI_TAPIVOT>(L, A.csr, x, y, e, f, gate);
        }
    }
    if (A.format == TACTA_CSR && A.csr.cfg.kind == 2) {
        switch (epi) {
        case EPI_NONE: return spmv_tiled_launch<EPI_NONE>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM: return spmv_tiled_launch<EPI_NORM>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID: return spmv_tiled_launch<EPI_RESID>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID_F32: return spmv_tiled_launch<EPI_RESID_F32>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM_POS: return spmv_tiled_launch<EPI_NORM_POS>(L, A.csr, x, y, e, f, gate);
        default: return spmv_tiled_launch<EPI_TAPIVOT>(L, A.csr, x, y, e, f, gate);
        }
    }
    if (A.format == TACTA_CSR) {
        CsrAcc acc{A.csr.rowptr, A.csr.colidx, A.csr.vals, A.csr.rows};
        return spmv_dispatch(L, A.csr.cfg.kind, acc, x, y, epi, e, f, gate);
    }
    switch (epi) {
    case EPI_NONE: return dense_launch<EPI_NONE>(L, A.dense, x, y, e, f, gate);
    case EPI_NORM: return dense_launch<EPI_NORM>(L, A.dense, x, y, e, f, gate);
    case EPI_RESID: return dense_launch<EPI_RESID>(L, A.dense, x, y, e, f, gate);
    case EPI_RESID_F32: return dense_launch<EPI_RESID_F32>(L, A.dense, x, y, e, f, gate);
    case EPI_NORM_POS: return dense_launch<EPI_NORM_POS>(L, A.dense, x, y, e, f, gate);
    default: return dense_launch<EPI_TAPIVOT>(L, A.dense, x, y, e, f, gate);
    }
}

// ------------------------------------------------------------------ vector kernels

struct VecPtrs { double* p[kTMax]; };
struct F32Ptrs { float* p[kTMax]; };

// CTA update (Eqs. CTAGEN7, CTAGEN7A): x += sum alpha_i z_i, r -= sum alpha_i u_i, ||r||².
template <int T>
__global__ void __launch_bounds__(kBlock)
cta_update(int64_t m, int64_t n, double* __restrict__ x, double* __restrict__ r, VecPtrs z,
           VecPtrs u, Ctl* ctl, double* partials, FinArgs f) {
    const int64_t len = m > n ? m : n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int32_t status = ctl->status;   // loaded together with alpha
    double al[T];
#pragma unroll
    for (int j = 0; j < T; ++j) al[j] = ctl->alpha[j];
    if (status != 0) return;
    double a0 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        if (i < n) {
            double v = x[i];
#pragma unroll
            for (int j = 0; j < T; ++j) v = fma(al[j], __ldg(z.p[j] + i), v);
            x[i] = v;
        }
        if (i < m) {
            double v = r[i];
#pragma unroll
            for (int j = 0; j < T; ++j) v = fma(-al[j], __ldg(u.p[j] + i), v);
            r[i] = v;
            a0 = fma(v, v, a0);
        }
    }
    reduce_and_finish<1, kBlock, true>(a0, 0.0, ctl, partials, f);
}

// TA update (Alg. 2.2): b'' = (1-alpha) b' + alpha v, i.e. with d = b - b' and the stored
// w = v - b', d'' = d - alpha w (one FMA per entry: the FP64 pipe, not HBM, bounds this
// kernel on GB300); x'' = (1-alpha) x + (alpha s) c; reductions ||d||², dᵀb for the next
// iteration.
__global__ void __launch_bounds__(kBlock)
ta_update(int64_t m, int64_t n, double* __restrict__ x, double* __restrict__ d,
          const double* __restrict__ b, const double* __restrict__ w, const double* __restrict__ c,
          Ctl* ctl, double* partials, FinArgs f) {
    if (ctl->status != 0) return;
    if (!ctl->pivot) {   // rho grew: nothing moves, only the bookkeeping
        if (blockIdx.x == 0 && threadIdx.x == 0) finish(ctl, f, ctl->rn2, ctl->db);
        return;
    }
    const double al = ctl->ta_alpha;
    const double as = al * ctl->s;
    const double om = 1.0 - al;
    double a0 = 0.0, a1 = 0.0;
    const int64_t len = m > n ? m : n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        if (i < m) {
            const double bv = __ldg(b + i);
            const double dv = fma(-al, __ldg(w + i), d[i]);
            d[i] = dv;
            a0 = fma(dv, dv, a0);
            a1 = fma(dv, bv, a1);
        }
        if (i < n) x[i] = om * x[i] + as * __ldg(c + i);
    }
    reduce_and_finish<2, kBlock, true>(a0, a1, ctl, partials, f);
}

// sum a_i² and sum a_i b_i (b may be null) over one vector, with a finisher.
__global__ void __launch_bounds__(kBlock)
reduce_vec(int64_t len, const double* __restrict__ a, const double* __restrict__ b, Ctl* ctl,
           double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    double a0 = 0.0, a1 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const double v = __ldg(a + i);
        a0 = fma(v, v, a0);
        if (b) a1 = fma(v, __ldg(b + i), a1);
    }
    reduce_and_finish(a0, a1, ctl, partials, f);
}

__global__ void copy_gated(double* __restrict__ dst, const double* __restrict__ src, int64_t len,
                           const Ctl* ctl, int gate) {
    if (gated_out(ctl, gate)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride)
        dst[i] = src[i];
}

__global__ void fill_kernel(double* __restrict__ dst, double v, int64_t len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) dst[i] = v;
}

// ------------------------------------------------------------------ mixed precision: FP32 chain
//
// The matrix values and the chain vectors z_i, u_i, r are FP32 (half the bytes,
// and FP32 FMAs run at ~60x the FP64 rate on GB300). Products accumulate in
// FP32; each thread's share of a moment (sum of y² over its rows) is kept in
// FP32 and the block / grid sums are FP64. The auxiliary solve, the stop tests
// and every scalar stay FP64 in the finishers; the true residual b - A x is
// computed by the FP64 product (refinement) every R steps and at stop checks.

template <int CAP, bool XW>
struct __align__(16) TileStage32 {
    float vals[CAP + 4];
    int32_t cols[CAP + 4];
    int32_t rp[kTileRows + 8];
    float xs[XW ? kXSpan + 4 : 4];
};

template <int CAP, bool XW>
size_t spmv32_smem() { return 2 * sizeof(TileStage32<CAP, XW>); }

template <int CAP, bool XW>
__device__ __forceinline__ void tile_issue32(const int4 d, const int2 w, TileStage32<CAP, XW>* st,
                                             uint64_t* bar, const int32_t* rowptr,
                                             const int32_t* colidx, const float* vals, const float* x) {
    const int a0 = d.z & ~3, c0 = d.z & ~3, r0 = d.x & ~3;
    const uint32_t bv = d.w > d.z ? round16((uint32_t)(d.w - a0) * 4u) : 0u;
    const uint32_t bc = d.w > d.z ? round16((uint32_t)(d.w - c0) * 4u) : 0u;
    const uint32_t br = round16((uint32_t)(d.y + 1 - r0) * 4u);
    uint32_t bx = 0;
    int x0 = 0;
    if (XW && d.w > d.z) {
        x0 = w.x & ~3;
        bx = round16((uint32_t)(w.y + 1 - x0) * 4u);
    }
    mbar_expect_tx(bar, bv + bc + br + bx);
    if (bv) bulk_g2s(st->vals, vals + a0, bv, bar);
    if (bc) bulk_g2s(st->cols, colidx + c0, bc, bar);
    bulk_g2s(st->rp, rowptr + r0, br, bar);
    if (bx) bulk_g2s(st->xs, x + x0, bx, bar);
}

template <int CAP, bool XW, int EPI>
__global__ void __launch_bounds__(kTileRows)
spmv32_tiled(const int4* __restrict__ tiles, const int2* __restrict__ xwin, int ntiles,
             const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
             const float* __restrict__ vals, const float* __restrict__ x, float* __restrict__ y,
             float scale, Ctl* ctl, double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileStage32<CAP, XW>* st = reinterpret_cast<TileStage32<CAP, XW>*>(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int failed;
    const int tid = threadIdx.x;
    const int G = gridDim.x;
    const int2 nowin = make_int2(0, 0);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        for (int j = 0; j < 2; ++j) {
            const int t = blockIdx.x + j * G;
            if (t < ntiles)
                tile_issue32<CAP, XW>(__ldg(tiles + t), XW ? __ldg(xwin + t) : nowin, st + j, bar + j,
                                      rowptr, colidx, vals, x);
        }
    }
    __syncthreads();
    float acc = 0.0f;
    for (int j = 0;; ++j) {
        const int t = blockIdx.x + j * G;
        if (t >= ntiles) break;
        const int sidx = j & 1;
        const int4 d = __ldg(tiles + t);
        const int xw0 = XW ? (__ldg(&xwin[t].x) & ~3) : 0;
        const bool ok = !failed && mbar_wait_bounded(bar + sidx, (uint32_t)((j >> 1) & 1));
        if (!ok) {
            failed = 1;
            atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
        }
        const TileStage32<CAP, XW>* S = st + sidx;
        const int row = d.x + tid;
        const bool active = ok && row < d.y;
        int kb = 0, len = 0;
        if (active) {
            const int r0 = d.x & ~3;
            kb = S->rp[row - r0];
            len = S->rp[row + 1 - r0] - kb;
        }
        const int vb = kb - (d.z & ~3);
        float sum = 0.0f;
        for (int u = 0; u < len; ++u) {
            const int c = S->cols[vb + u];
            const float xv = XW ? S->xs[c - xw0] : __ldg(x + c);
            sum = fmaf(S->vals[vb + u], xv, sum);
        }
        if (active) {
            sum *= scale;   // a power of two: exact
            y[row] = sum;
            if (EPI == EPI_NORM) acc = fmaf(sum, sum, acc);
        }
        __syncthreads();
        if (tid == 0 && !failed) {
            const int t2 = t + 2 * G;
            if (t2 < ntiles)
                tile_issue32<CAP, XW>(__ldg(tiles + t2), XW ? __ldg(xwin + t2) : nowin, st + sidx,
                                      bar + sidx, rowptr, colidx, vals, x);
        }
    }
    if (failed && tid == 0) {
        for (int j = 0; j < 2; ++j) mbar_wait_bounded(bar + j, 0u);
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<1>((double)acc, 0.0, ctl, partials, f);
}

// FP32 run-staged product, warp-specialised (the mixed-precision chain): the FP64
// operand's tiles, runs and 16-bit slots with the FP32 copy of the values; runs start
// and end on multiples of 4 entries, so the FP32 x runs move in 16-byte units too.
template <int EPI>
__global__ void __launch_bounds__(kRwThreads, kRw32BlocksPerSM)
spmv32_tiled_rw(const int4* __restrict__ tiles, const int2* __restrict__ runs, int ntiles,
                const int32_t* __restrict__ rowptr, const uint16_t* __restrict__ lcol,
                const float* __restrict__ vals, const float* __restrict__ x, float* __restrict__ y, float scale,
                Ctl* ctl, double* partials, FinArgs f, int gate) {
    constexpr int S = kRw32Stages;
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TileStageR32* st = reinterpret_cast<TileStageR32*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ volatile int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRwConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    __syncthreads();
    int last_use[S];
    for (int k = 0; k < S; ++k) last_use[k] = -1;
    float acc = 0.0f;
    if (warp == kRwConsumers) {
        TilePrefetch pf;
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles || __any_sync(0xffffffffu, failed != 0)) break;   // one decision per warp
            const TileMeta tm = pf.get(j, tiles, runs, ntiles, G, lane);
            if (lane == 0) {
                const int k = j % S, u = j / S;
                if (u > 0 && !mbar_wait_bounded(&empty[k], (uint32_t)((u - 1) & 1))) {
                    failed = 1;
                    atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                } else {
                    st[k].desc = tm.d;
                    tile_issue_r<float>(tm, st + k, &full[k], rowptr, lcol, vals, x);
                    last_use[k] = u;
                }
            }
            __syncwarp();
        }
    } else {
        for (int j = 0;; ++j) {
            const int t = blockIdx.x + j * G;
            if (t >= ntiles) break;
            const int k = j % S;
            const bool ok = !failed && mbar_wait_bounded(&full[k], (uint32_t)((j / S) & 1));
            if (!__all_sync(0xffffffffu, ok)) {   // the warp takes one path
                if (lane == 0) {
                    failed = 1;
                    atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                }
                break;
            }
            int row;
            bool active;
            float sum = rw_row_dot(st + k, warp, lane, row, active);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[k]);
            if (active) {
                sum *= scale;   // a power of two: exact
                y[row] = sum;
                if (EPI == EPI_NORM) acc = fmaf(sum, sum, acc);
            }
        }
    }
    __syncthreads();
    if (failed && warp == kRwConsumers && lane == 0) {
        for (int k = 0; k < S; ++k)
            if (last_use[k] >= 0) mbar_wait_bounded(&full[k], (uint32_t)(last_use[k] & 1));
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<1, kRwThreads>((double)acc, 0.0, ctl, partials, f);
}

// warp per row for long FP32 rows
template <int EPI>
__global__ void __launch_bounds__(kBlock)
spmv32_warp(int64_t rows, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
            const float* __restrict__ vals, const float* __restrict__ x, float* __restrict__ y,
            float scale, Ctl* ctl, double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    float acc = 0.0f;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        const int64_t b = __ldg(rowptr + row), en = __ldg(rowptr + row + 1);
        float sum = 0.0f;
        for (int64_t k = b + lane; k < en; k += 32) sum = fmaf(__ldg(vals + k), __ldg(x + __ldg(colidx + k)), sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (lane == 0) {
            sum *= scale;
            y[row] = sum;
            if (EPI == EPI_NORM) acc = fmaf(sum, sum, acc);
        }
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish<1>((double)acc, 0.0, ctl, partials, f);
}

template <int CAP, bool XW, int EPI>
static cudaError_t spmv32_tiled_launch(const LaunchCtx& L, const DevCSR32& A, const float* x, float* y,
                                       float scale, FinArgs f, int gate) {
    const DevCSR& a = *A.base;
    const size_t sm = spmv32_smem<CAP, XW>();
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(6, (220u << 10) / (sm + 3072)));
    const int grid = std::min(a.ntiles, std::max(1, (L.max_grid / 8) * per_sm));
    spmv32_tiled<CAP, XW, EPI><<<grid, kTileRows, sm, L.stream>>>(a.tiles, a.xwin, a.ntiles, a.rowptr,
                                                                   a.colidx, A.vals, x, y, scale, L.ctl,
                                                                   L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

template <int EPI>
static cudaError_t spmv32_epi(const LaunchCtx& L, const DevCSR32& A, const float* x, float* y, float scale,
                              FinArgs f, int gate) {
    const DevCSR& a = *A.base;
    if (a.cfg.kind == 3 && a.lcol) {
        static const char attr_key = 0;
        constexpr size_t sm = kRw32Stages * sizeof(TileStageR32);
        if (!done_on_device(&attr_key)) {
            const cudaError_t e2 = cudaFuncSetAttribute(spmv32_tiled_rw<EPI>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e2 != cudaSuccess) return e2;
            mark_done_on_device(&attr_key);
        }
        const int grid = std::min(a.ntiles, std::max(1, (L.max_grid / 8) * kRw32BlocksPerSM));
        spmv32_tiled_rw<EPI><<<grid, kRwThreads, sm, L.stream>>>(a.tiles, a.runs, a.ntiles, a.rowptr, a.lcol, A.vals,
                                                                 x, y, scale, L.ctl, L.partials, f, gate);
        if (L.launches) ++*L.launches;
        return cudaGetLastError();
    }
    if (a.cfg.kind == 3) return spmv32_tiled_launch<kTileCapSmall, true, EPI>(L, A, x, y, scale, f, gate);
    if (a.cfg.kind == 2) {
        if (a.cap <= kTileCapSmall)
            return spmv32_tiled_launch<kTileCapSmall, false, EPI>(L, A, x, y, scale, f, gate);
        return spmv32_tiled_launch<kTileCapLarge, false, EPI>(L, A, x, y, scale, f, gate);
    }
    spmv32_warp<EPI><<<L.max_grid, kBlock, 0, L.stream>>>(a.rows, a.rowptr, a.colidx, A.vals, x, y, scale,
                                                          L.ctl, L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_spmv32(const LaunchCtx& L, const DevCSR32& A, const float* x, float* y, float scale,
                          int epi, FinArgs f, int gate) {
    return epi == EPI_NORM ? spmv32_epi<EPI_NORM>(L, A, x, y, scale, f, gate)
                           : spmv32_epi<EPI_NONE>(L, A, x, y, scale, f, gate);
}

// max_i sum_k |A_ik| (the infinity norm), for the chain scale of the mixed path
__global__ void abs_row_sum_max_kernel(int64_t rows, const int32_t* __restrict__ rowptr,
                                       const double* __restrict__ vals, unsigned long long* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double best = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        double s = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += fabs(vals[k]);
        best = fmax(best, s);
    }
    // non-negative doubles order like their bit patterns
    atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

cudaError_t abs_row_sum_max(cudaStream_t s, const DevCSR& A, double* dev_out, double* host_out) {
    cudaError_t e = cudaMemsetAsync(dev_out, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    abs_row_sum_max_kernel<<<1024, kBlock, 0, s>>>(A.rows, A.rowptr, A.vals,
                                                   reinterpret_cast<unsigned long long*>(dev_out));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(host_out, dev_out, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

// Dense FP32 product of the mixed-precision chain: y = (A x) * scale for row-major A,
// ||y||² (FP64, added per row) to the finisher. WPR warps share a row (the grid then has
// enough warps in flight for HBM when rows are few and long). When the rows are 16-byte
// aligned, x is staged in shared memory once per block and each lane keeps eight 16-byte
// loads of A in flight (registers hold A only), summing an interleaved share of the row's
// vectors with four independent accumulators; the WPR partial sums meet in shared memory
// in warp order (deterministic).
constexpr int kDenseXSmem = 64 * 1024;   // x staged in shared memory up to 16,384 columns

template <int WPR>
__global__ void __launch_bounds__(kBlock)
dense32_rows(int64_t rows, int64_t cols, const float* __restrict__ A, const float* __restrict__ x,
             float* __restrict__ y, float scale, Ctl* ctl, double* partials, FinArgs f, int gate) {
    if (gated_out(ctl, gate)) return;
    if (gate != GATE_FORCE && blockIdx.x == 0 && threadIdx.x == 0) ctl->matvecs += 1;
    constexpr int RPB = (kBlock / 32) / WPR;   // rows per block and pass
    extern __shared__ float4 xs[];             // x (staged: cols / 4 vectors)
    __shared__ float red[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rl = warp / WPR, part = warp % WPR;
    const bool vec = (cols & 3) == 0;          // rows start 16-byte aligned
    const int64_t nv = cols >> 2;
    const bool staged = vec && cols * 4 <= kDenseXSmem;
    const int64_t step = 32 * WPR;
    const int64_t groups = (rows + RPB - 1) / RPB;
    // eight 16-byte loads of A per lane and chunk, predicated at the row's end so that a
    // chunk always has all its loads in flight; the first chunk of the block's first row
    // is issued before x is staged, so the staging overlaps the first loads
    float4 p[8];
    auto load_chunk = [&](int64_t row, int64_t c0) {
        const float4* a4 = reinterpret_cast<const float4*>(A + row * cols);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t idx = c0 + k * step;
            p[k] = (row < rows && idx < nv) ? __ldcs(a4 + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if (staged) {
        if ((int64_t)blockIdx.x < groups) load_chunk(blockIdx.x * RPB + rl, part * 32 + lane);
        const float4* x4 = reinterpret_cast<const float4*>(x);
        for (int64_t i = threadIdx.x; i < nv; i += kBlock) xs[i] = __ldg(x4 + i);
        __syncthreads();
    }
    double a0 = 0.0;
    for (int64_t gidx = blockIdx.x; gidx < groups; gidx += gridDim.x) {
        const int64_t row = gidx * RPB + rl;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        if (staged) {
            for (int64_t c0 = part * 32 + lane; c0 < nv; c0 += 8 * step) {
                if (!(gidx == (int64_t)blockIdx.x && c0 == part * 32 + lane)) load_chunk(row, c0);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int64_t idx = c0 + k * step;
                    if (idx < nv) {
                        const float4 q = xs[idx];
                        s0 = fmaf(p[k].x, q.x, s0); s1 = fmaf(p[k].y, q.y, s1);
                        s2 = fmaf(p[k].z, q.z, s2); s3 = fmaf(p[k].w, q.w, s3);
                    }
                }
            }
        } else if (row < rows) {
            const float* a = A + row * cols;
            for (int64_t c = part * 32 + lane; c < cols; c += step) s0 = fmaf(__ldg(a + c), __ldg(x + c), s0);
        }
        float sum = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (WPR == 1) {
            if (lane == 0 && row < rows) {
                const float v = sum * scale;
                y[row] = v;
                a0 = fma((double)v, (double)v, a0);
            }
        } else {
            if (lane == 0) red[warp] = sum;
            __syncthreads();
            if (part == 0 && lane == 0 && row < rows) {
                float t = red[warp];
                for (int q = 1; q < WPR; ++q) t += red[warp + q];
                const float v = t * scale;
                y[row] = v;
                a0 = fma((double)v, (double)v, a0);
            }
            __syncthreads();
        }
    }
    reduce_and_finish<1>(a0, 0.0, ctl, partials, f);
}

cudaError_t dense32_prepare() {
    static const char done_key = 0;
    if (done_on_device(&done_key)) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (const void* k : {(const void*)dense32_rows<1>, (const void*)dense32_rows<2>, (const void*)dense32_rows<4>,
                          (const void*)dense32_rows<8>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseXSmem);
    if (e == cudaSuccess) mark_done_on_device(&done_key);
    return e;
}

cudaError_t launch_dense32(const LaunchCtx& L, int64_t rows, int64_t cols, const float* A, const float* x,
                           float* y, float scale, FinArgs f, int gate) {
    cudaError_t e = dense32_prepare();
    if (e != cudaSuccess) return e;
    const size_t sm = ((cols & 3) == 0 && cols * 4 <= kDenseXSmem) ? (size_t)cols * 4 : 0;
    // one wave of resident blocks looping over row groups of 8 / wpr rows; wpr is the split
    // whose groups fill the wave most evenly (the busiest block takes ceil(groups / wave))
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, dense32_rows<4>, kBlock, sm) != cudaSuccess || per < 1)
        per = 1;
    const int wave = std::min(L.max_grid, per * (L.max_grid / 8));
    int wpr = 1;
    double best = -1.0;
    for (int w = 1; w <= 8; w *= 2) {
        if (w > 1 && cols < 512LL * w) break;
        const double groups = (double)((rows * w + (kBlock / 32) - 1) / (kBlock / 32));
        const double eff = groups < wave ? groups / wave : (groups / wave) / std::ceil(groups / wave);
        if (eff > best + 1e-9) { best = eff; wpr = w; }
    }
    const int64_t rpb = (kBlock / 32) / wpr;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows + rpb - 1) / rpb, (int64_t)wave));
    if (L.launches) ++*L.launches;
    switch (wpr) {
    case 1: dense32_rows<1><<<grid, kBlock, sm, L.stream>>>(rows, cols, A, x, y, scale, L.ctl, L.partials, f, gate); break;
    case 2: dense32_rows<2><<<grid, kBlock, sm, L.stream>>>(rows, cols, A, x, y, scale, L.ctl, L.partials, f, gate); break;
    case 4: dense32_rows<4><<<grid, kBlock, sm, L.stream>>>(rows, cols, A, x, y, scale, L.ctl, L.partials, f, gate); break;
    default: dense32_rows<8><<<grid, kBlock, sm, L.stream>>>(rows, cols, A, x, y, scale, L.ctl, L.partials, f, gate); break;
    }
    return cudaGetLastError();
}

// max_i sum_k |A_ik| of a dense row-major matrix (the infinity norm)
__global__ void dense_abs_row_sum_max_kernel(int64_t rows, int64_t cols, const double* __restrict__ vals,
                                             unsigned long long* out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double best = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        double sm = 0.0;
        for (int64_t c = lane; c < cols; c += 32) sm += fabs(vals[r * cols + c]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
        best = fmax(best, sm);
    }
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

cudaError_t dense_abs_row_sum_max(cudaStream_t s, int64_t rows, int64_t cols, const double* vals, double* dev_out,
                                  double* host_out) {
    cudaError_t e = cudaMemsetAsync(dev_out, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    dense_abs_row_sum_max_kernel<<<1024, kBlock, 0, s>>>(rows, cols, vals,
                                                         reinterpret_cast<unsigned long long*>(dev_out));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(host_out, dev_out, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t spmv32_prepare() {
    static const char done_key = 0;
    if (done_on_device(&done_key)) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define TACTA_S32_ATTR(CAP, XW, EPI)                                                                        \
    if (e == cudaSuccess)                                                                                   \
        e = cudaFuncSetAttribute(spmv32_tiled<CAP, XW, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)spmv32_smem<CAP, XW>());
    TACTA_S32_ATTR(kTileCapSmall, true, EPI_NORM) TACTA_S32_ATTR(kTileCapSmall, true, EPI_NONE)
    TACTA_S32_ATTR(kTileCapSmall, false, EPI_NORM) TACTA_S32_ATTR(kTileCapSmall, false, EPI_NONE)
    TACTA_S32_ATTR(kTileCapLarge, false, EPI_NORM) TACTA_S32_ATTR(kTileCapLarge, false, EPI_NONE)
#undef TACTA_S32_ATTR
    if (e == cudaSuccess) mark_done_on_device(&done_key);
    return e;
}

// CTA update in FP32: dx += sum alpha_i z_i (the correction to the FP64 x since the
// last refinement), r -= sum alpha_i u_i; ||r||² per thread in FP32, reduced in FP64.
template <int T>
__global__ void __launch_bounds__(kBlock)
cta_update32(int64_t m, int64_t n, float* __restrict__ dx, float* __restrict__ r, F32Ptrs z, F32Ptrs u,
             float xscale, Ctl* ctl, double* partials, FinArgs f) {
    const int64_t len = m > n ? m : n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (ctl->status != 0) return;
    // the chain vectors are scaled (z_i by s^(2i-1), u_i by s^(2i), s = xscale a power of
    // two), so the solve on the scaled moments gives beta with x += s sum beta_i z_i,
    // r -= sum beta_i u_i
    float al[T], ax[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
        al[j] = (float)ctl->alpha[j];
        ax[j] = (float)(ctl->alpha[j] * (double)xscale);
    }
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        if (i < n) {
            float v = dx[i];
#pragma unroll
            for (int j = 0; j < T; ++j) v = fmaf(ax[j], __ldg(z.p[j] + i), v);
            dx[i] = v;
        }
        if (i < m) {
            float v = r[i];
#pragma unroll
            for (int j = 0; j < T; ++j) v = fmaf(-al[j], __ldg(u.p[j] + i), v);
            r[i] = v;
            acc = fmaf(v, v, acc);
        }
    }
    reduce_and_finish<1, kBlock, true>((double)acc, 0.0, ctl, partials, f);
}

__global__ void loop_begin_kernel(Ctl* ctl, int32_t limit) {
    ctl->loops = 0;
    ctl->loop_limit = limit;
}

__global__ void loop_continue_kernel(Ctl* ctl, cudaGraphConditionalHandle h) {
    const int32_t n = ++ctl->loops;
    cudaGraphSetConditional(h, (ctl->status == 0 && n < ctl->loop_limit) ? 1u : 0u);
}

cudaError_t launch_loop_begin(cudaStream_t s, Ctl* ctl, int32_t limit) {
    loop_begin_kernel<<<1, 1, 0, s>>>(ctl, limit);
    return cudaGetLastError();
}

cudaError_t launch_loop_continue(cudaStream_t s, Ctl* ctl, cudaGraphConditionalHandle h) {
    loop_continue_kernel<<<1, 1, 0, s>>>(ctl, h);
    return cudaGetLastError();
}

// x += (double) dx, dx = 0: the FP32 correction folded into the FP64 iterate
__global__ void fold_correction(int64_t n, double* __restrict__ x, float* __restrict__ dx, const Ctl* ctl,
                                int gate) {
    if (gated_out(ctl, gate)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        x[i] += (double)dx[i];
        dx[i] = 0.0f;
    }
}

__global__ void d2f_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) dst[i] = (float)src[i];
}

cudaError_t launch_cta_update32(const LaunchCtx& L, int t, int64_t m, int64_t n, float* dx, float* r,
                                float* const* z, float* const* u, float xscale, FinArgs f) {
    F32Ptrs zp{}, up{};
    for (int j = 0; j < t; ++j) { zp.p[j] = z[j]; up.p[j] = u[j]; }
    const int g = L.max_grid;
    switch (t) {
    case 1: cta_update32<1><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    case 2: cta_update32<2><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    case 3: cta_update32<3><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    case 4: cta_update32<4><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    case 5: cta_update32<5><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    case 6: cta_update32<6><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    case 7: cta_update32<7><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    default: cta_update32<8><<<g, kBlock, 0, L.stream>>>(m, n, dx, r, zp, up, xscale, L.ctl, L.partials, f); break;
    }
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_fold_correction(const LaunchCtx& L, int64_t n, double* x, float* dx, int gate) {
    fold_correction<<<L.max_grid, kBlock, 0, L.stream>>>(n, x, dx, L.ctl, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t convert_to_f32(cudaStream_t s, const double* src, float* dst, int64_t len) {
    int64_t blocks = (len + kBlock - 1) / kBlock;
    if (blocks < 1) blocks = 1;
    if (blocks > 65536) blocks = 65536;
    d2f_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(src, dst, len);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pattern outer product
// out[k] += alpha u[row(k)] v[col(k)] over the stored entries of A (CSR: nonzero order;
// dense: row-major) -- the gradient dL/dA of a linear solve restricted to A's pattern.
__global__ void __launch_bounds__(kBlock)
outer_on_pattern_csr(int64_t rows, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                     double alpha, const double* __restrict__ u, const double* __restrict__ v,
                     double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const double au = alpha * u[r];
        for (int64_t k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) out[k] = fma(au, v[colidx[k]], out[k]);
    }
}

__global__ void __launch_bounds__(kBlock)
outer_on_pattern_dense(int64_t rows, int64_t cols, double alpha, const double* __restrict__ u,
                       const double* __restrict__ v, double* __restrict__ out) {
    const int64_t total = rows * cols;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride) {
        const int64_t r = k / cols, c = k - r * cols;
        out[k] = fma(alpha * u[r], v[c], out[k]);
    }
}

cudaError_t launch_outer_on_pattern(cudaStream_t s, int grid, const DevOperand& A, double alpha, const double* u,
                                    const double* v, double* out) {
    if (A.format == TACTA_CSR)
        outer_on_pattern_csr<<<grid, kBlock, 0, s>>>(A.csr.rows, A.csr.rowptr, A.csr.colidx, alpha, u, v, out);
    else
        outer_on_pattern_dense<<<grid, kBlock, 0, s>>>(A.dense.rows, A.dense.cols, alpha, u, v, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_cta_update(const LaunchCtx& L, int t, int64_t m, int64_t n, double* x,
                              double* r, double* const* z, double* const* u, FinArgs f) {
    VecPtrs zp{}, up{};
    for (int j = 0; j < t; ++j) { zp.p[j] = z[j]; up.p[j] = u[j]; }
    const int g = L.max_grid;
    switch (t) {
    case 1: cta_update<1><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    case 2: cta_update<2><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    case 3: cta_update<3><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    case 4: cta_update<4><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    case 5: cta_update<5><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    case 6: cta_update<6><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    case 7: cta_update<7><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    default: cta_update<8><<<g, kBlock, 0, L.stream>>>(m, n, x, r, zp, up, L.ctl, L.partials, f); break;
    }
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_ta_update(const LaunchCtx& L, int64_t m, int64_t n, double* x, double* d,
                             const double* b, const double* v, const double* c, FinArgs f) {
    ta_update<<<L.max_grid, kBlock, 0, L.stream>>>(m, n, x, d, b, v, c, L.ctl, L.partials, f);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_reduce_vec(const LaunchCtx& L, int64_t len, const double* a, const double* b,
                              FinArgs f, int gate) {
    reduce_vec<<<L.max_grid, kBlock, 0, L.stream>>>(len, a, b, L.ctl, L.partials, f, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

cudaError_t launch_ctl_init(const LaunchCtx& L, const Ctl& host_init) {
    // the control block is plain data: one async copy from a host staging struct
    // (the caller keeps host_init alive until the stream has consumed it)
    return cudaMemcpyAsync(L.ctl, &host_init, sizeof(Ctl), cudaMemcpyHostToDevice, L.stream);
}

cudaError_t launch_copy_gated(const LaunchCtx& L, double* dst, const double* src, int64_t len,
                              int gate) {
    copy_gated<<<L.max_grid, kBlock, 0, L.stream>>>(dst, src, len, L.ctl, gate);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

// CTA step decision (Alg. 1.1 with Eq. eqcoeff), one thread, after the chain's last
// product: finite moments, the normal-equation test, the auxiliary solve -> alpha. It is
// its own kernel so that the solve's registers (its arrays live in registers) do not
// count against the occupancy of every product and update kernel, as they would if it
// ran inside their shared finisher.
// The step decision and auxiliary solve (one thread, FP64), in its own kernel so that
// the solve's registers stay out of the streaming kernels. The control block is staged
// in shared memory by all threads at once, so the one-thread solve works on shared-
// memory loads instead of a chain of dependent global loads.
__global__ void __launch_bounds__(384) cta_aux_step(Ctl* c, int t, const double* part, int G) {
    __shared__ Ctl sc;
    static_assert(sizeof(Ctl) % 8 == 0, "the control block copies as 8-byte words");
    {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(c);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sc);
        for (int i = threadIdx.x; i < (int)(sizeof(Ctl) / 8); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (part != nullptr && threadIdx.x == 0) c->chain_bar = 0;   // the fused chain's counter starts over
    if (sc.status != 0) return;
    if (part != nullptr) sum_moment_partials(&sc, t, part, G, c);   // fused chain: the moments' partials
    if (threadIdx.x != 0) return;
    const int status = aux_decide(&sc, t);
    if (status != 0 && !sc.enh_stop) {
        c->status = status;
        return;
    }
    for (int k = 0; k < t; ++k) c->alpha[k] = sc.alpha[k];
    c->rank = sc.rank;
    if (sc.enh_stop) c->enh_stop = 1;
}

cudaError_t launch_cta_aux_step(const LaunchCtx& L, int t, const double* part, int G) {
    // 12 warps for the moment sums: the solve's registers (~134 per thread) allow 384 threads
    cta_aux_step<<<1, part ? 384 : 32, 0, L.stream>>>(L.ctl, t, part, G);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

__global__ void hist_sqrt(double* h, int64_t len) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        h[i] = sqrt(h[i]);
}

cudaError_t launch_hist_sqrt(cudaStream_t s, double* h, int64_t len) {
    if (len <= 0) return cudaSuccess;
    hist_sqrt<<<(int)std::min<int64_t>((len + kBlock - 1) / kBlock, 1024), kBlock, 0, s>>>(h, len);
    return cudaGetLastError();
}

cudaError_t launch_fill(const LaunchCtx& L, double* dst, double v, int64_t len) {
    fill_kernel<<<L.max_grid, kBlock, 0, L.stream>>>(dst, v, len);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

}  // namespace tacta
