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

namespace tacta {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ bool gated_out(const Ctl* c, int gate) {
    if (gate == GATE_FORCE) return false;
    if (c->status != 0) return true;
    if (gate == GATE_NEED_TRUE && !c->need_true) return true;
    if (gate == GATE_PIVOT && !c->pivot) return true;
    return false;
}

__device__ __forceinline__ bool finite(double v) { return v == v && fabs(v) <= DBL_MAX; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ finisher (one thread)

// Stop tests at the top of the loop of Alg. 1.1 / 2.1 / 2.2 (relative forms):
// residual passes on the true residual -> stop; on the recursive one -> ask for
// the true residual first; else the iteration cap.
__device__ void loop_top(Ctl* c) {
    if (!finite(c->rn2)) { c->status = TACTA_REASON_NONFINITE; return; }
    if (c->rn2 <= c->res_thr) {
        if (c->is_true) { c->status = TACTA_REASON_RESIDUAL; return; }
        c->need_true = 1;
        return;
    }
    if (c->k >= c->max_iter) c->status = TACTA_REASON_MAXITER;
}

__device__ void put_hist(Ctl* c, double* h) {
    if (h != nullptr && c->k < c->hist_cap) {
        h[c->k] = sqrt(c->rn2 / c->bn2);
        if (c->k + 1 > c->hist_len) c->hist_len = c->k + 1;
    }
}

// Auxiliary equation of order t (Eq. eqcoeff): [phi_{i+j}] alpha = [phi_i].
// Jacobi-scaled Cholesky in natural order, truncated at the first pivot
// <= pivot_tol; the leading block is solved and the trailing alphas are 0.
// Arithmetic uses explicit round-to-nearest operations (no contraction).
__device__ int hankel_solve_dev(const double* phi, int t, double pivot_tol, double* alpha) {
    double s[kTMax], G[kTMax][kTMax], L[kTMax][kTMax], y[kTMax], beta[kTMax];
    int tt = 0;
    for (int i = 1; i <= t; ++i) {
        if (!(phi[2 * i] > 0.0)) break;
        s[i - 1] = __ddiv_rn(1.0, __dsqrt_rn(phi[2 * i]));
        tt = i;
    }
    for (int i = 0; i < tt; ++i)
        for (int j = 0; j < tt; ++j) G[i][j] = __dmul_rn(__dmul_rn(s[i], phi[i + j + 2]), s[j]);
    int rank = 0;
    for (int k = 0; k < tt; ++k) {
        double d = G[k][k];
        for (int j = 0; j < k; ++j) d = __dsub_rn(d, __dmul_rn(L[k][j], L[k][j]));
        if (!(d > pivot_tol)) break;
        L[k][k] = __dsqrt_rn(d);
        for (int i = k + 1; i < tt; ++i) {
            double v = G[i][k];
            for (int j = 0; j < k; ++j) v = __dsub_rn(v, __dmul_rn(L[i][j], L[k][j]));
            L[i][k] = __ddiv_rn(v, L[k][k]);
        }
        rank = k + 1;
    }
    for (int i = 0; i < rank; ++i) {
        double v = __dmul_rn(s[i], phi[i + 1]);
        for (int j = 0; j < i; ++j) v = __dsub_rn(v, __dmul_rn(L[i][j], y[j]));
        y[i] = __ddiv_rn(v, L[i][i]);
    }
    for (int i = rank - 1; i >= 0; --i) {
        double v = y[i];
        for (int j = i + 1; j < rank; ++j) v = __dsub_rn(v, __dmul_rn(L[j][i], beta[j]));
        beta[i] = __ddiv_rn(v, L[i][i]);
    }
    for (int i = 0; i < t; ++i) alpha[i] = i < rank ? __dmul_rn(s[i], beta[i]) : 0.0;
    return rank;
}

__device__ __noinline__ void finish(Ctl* c, const FinArgs& f, double r0, double r1) {
    if (c->status == TACTA_REASON_TIMEOUT) return;   // a kernel gave up waiting: keep that verdict
    switch (f.kind) {
    case FIN_STORE:
        c->red[f.idx] = r0;
        c->red[f.idx + 1] = r1;
        break;
    case FIN_PHI:
        c->phi[f.idx] = r0;
        break;
    case FIN_CTA_STEP: {
        const int t = f.idx;
        c->phi[2 * t] = r0;
        for (int i = 1; i <= 2 * t; ++i)
            if (!finite(c->phi[i])) { c->status = TACTA_REASON_NONFINITE; return; }
        if (c->phi[1] <= c->nrm_thr) { c->status = TACTA_REASON_NORMAL; return; }
        c->rank = hankel_solve_dev(c->phi, t, c->pivot_tol, c->alpha);
        if (c->rank == 0) c->status = TACTA_REASON_BREAKDOWN;
        break;
    }
    case FIN_CTA_UPDATE:
        c->k += 1;
        c->is_true = 0;
        c->rn2 = r0;
        put_hist(c, f.hist);
        if (c->R > 0 && c->k % c->R == 0) { c->need_true = 1; break; }
        loop_top(c);
        break;
    case FIN_TRUE_RES:
        c->rn2 = r0;
        c->db = r1;
        c->is_true = 1;
        c->need_true = 0;
        put_hist(c, f.hist);
        loop_top(c);
        break;
    case FIN_TRIP_START:
        c->k = 0;
        c->rn2 = r0;
        c->db = r1;
        c->is_true = 1;
        c->need_true = 0;
        c->pivot = 0;
        put_hist(c, f.hist);
        loop_top(c);
        break;
    case FIN_TA_C: {
        c->cn2 = r0;
        if (!finite(r0) || !finite(c->db)) { c->status = TACTA_REASON_NONFINITE; return; }
        if (r0 <= c->nrm_thr) { c->status = TACTA_REASON_NORMAL; return; }
        const double cn = __dsqrt_rn(r0);
        if (__dmul_rn(c->rho, cn) >= c->db) {            // strict pivot (Eq. eqlem2)
            c->pivot = 1;
            c->s = __ddiv_rn(c->rho, cn);
        } else {
            c->pivot = 0;
            if (c->grow_rho) c->rho = fmax(__dmul_rn(2.0, c->rho), __ddiv_rn(c->db, cn));
            else c->status = TACTA_REASON_WITNESS;      // Alg. 2.1 STOP
        }
        break;
    }
    case FIN_TA_V:
        if (!(r1 > 0.0)) { c->status = TACTA_REASON_BREAKDOWN; return; }
        c->ta_alpha = fmin(__ddiv_rn(r0, r1), 1.0);
        break;
    case FIN_TA_UPDATE:
        c->k += 1;
        c->is_true = 0;
        if (c->pivot) { c->rn2 = r0; c->db = r1; }
        put_hist(c, f.hist);
        if (c->R > 0 && c->k % c->R == 0) { c->need_true = 1; break; }
        loop_top(c);
        break;
    case FIN_SETUP_B:
        c->bn2 = r0;
        if (r0 == 0.0) c->status = TACTA_REASON_ZERO_RHS;
        else if (!finite(r0)) c->status = TACTA_REASON_NONFINITE;
        break;
    case FIN_SETUP_MTB:
        c->mtbn2 = r0;
        c->res_thr = __dmul_rn(c->tol2, c->bn2);
        c->nrm_thr = __dmul_rn(c->tol_n2, r0);
        if (!finite(r0)) c->status = TACTA_REASON_NONFINITE;
        break;
    case FIN_SETUP_RHO:
        c->rho = __dsqrt_rn(r0);
        break;
    default:
        break;
    }
}

// Block-level reduction of (a0, a1), partial per block, last block sums all
// partials in fixed order and runs the finisher.
__device__ void reduce_and_finish(double a0, double a1, Ctl* ctl, double* partials,
                                  const FinArgs& f) {
    __shared__ double sh0[kBlock / 32], sh1[kBlock / 32];
    __shared__ int am_last;
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh0[w] = a0; sh1[w] = a1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { s0 += sh0[i]; s1 += sh1[i]; }
        partials[2 * blockIdx.x] = s0;
        partials[2 * blockIdx.x + 1] = s1;
        __threadfence();
        const unsigned ticket = atomicAdd(&ctl->counter, 1u);
        am_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        s0 += __ldcg(&partials[2 * i]);
        s1 += __ldcg(&partials[2 * i + 1]);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    __syncthreads();
    if (l == 0) { sh0[w] = s0; sh1[w] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { t0 += sh0[i]; t1 += sh1[i]; }
        ctl->counter = 0;
        finish(ctl, f, t0, t1);
    }
}

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

struct DenseAcc {
    const double* __restrict__ vals;
    int64_t rows, cols;
    __device__ __forceinline__ int64_t begin(int64_t r) const { return r * cols; }
    __device__ __forceinline__ int64_t end(int64_t r) const { return r * cols + cols; }
    __device__ __forceinline__ int64_t col(int64_t k, int64_t b) const { return k - b; }
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
    } else if (EPI == EPI_RESID) {
        const double bv = __ldg(e.b + row);
        const double v = bv - sum;
        y[row] = v;
        a0 = fma(v, v, a0);
        a1 = fma(v, bv, a1);
    } else {  // EPI_TAPIVOT: v = s (A c); w = v - b' = v - b + d
        const double v = s * sum;
        const double dv = __ldg(e.d + row);
        const double w = (v - __ldg(e.b + row)) + dv;
        y[row] = v;
        a0 = fma(dv, w, a0);
        a1 = fma(w, w, a1);
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
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish(a0, a1, ctl, partials, f);
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
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish(a0, a1, ctl, partials, f);
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

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait: gives up after ~2^31 SM cycles (about a second)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    return true;
}

template <int CAP>
struct __align__(16) TileStage {
    double vals[CAP + 2];
    int32_t cols[CAP + 4];
    int32_t rp[kTileRows + 8];
};

size_t spmv_tiled_smem(int cap) {
    return cap <= kTileCapSmall ? 2 * sizeof(TileStage<kTileCapSmall>) : 2 * sizeof(TileStage<kTileCapLarge>);
}

__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

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
    for (int j = 0;; ++j) {
        const int t = blockIdx.x + j * G;
        if (t >= ntiles) break;
        const int sidx = j & 1;
        const int4 d = __ldg(tiles + t);
        bool ok = !failed && mbar_wait_bounded(bar + sidx, (uint32_t)((j >> 1) & 1));
        if (!ok) {
            failed = 1;
            atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
        }
        const TileStage<CAP>* S = st + sidx;
        const int row = d.x + tid;
        const bool active = ok && row < d.y;
        int kb = 0, len = 0;
        if (active) {
            const int r0 = d.x & ~3;
            kb = S->rp[row - r0];
            len = S->rp[row + 1 - r0] - kb;
        }
        // A predicated-off FP64 FMA still occupies the narrow FP64 pipe, so each warp
        // issues exactly max(row length over its lanes) FMAs, in groups of 8 with all
        // gathers of a group in flight before its FMA chain.
        const int maxlen = __reduce_max_sync(0xffffffffu, len);
        double sum = 0.0;
        const double* vp = S->vals + (kb - (d.z & ~1));
        const int32_t* cp = S->cols + (kb - (d.z & ~3));
        for (int u0 = 0; u0 < maxlen; u0 += 8) {
            double xv[8], vv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (u0 + u < len) {
                    xv[u] = __ldg(x + cp[u0 + u]);
                    vv[u] = vp[u0 + u];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (u0 + u >= maxlen) break;   // warp-uniform
                if (u0 + u < len) sum = fma(vv[u], xv[u], sum);
            }
        }
        if (active) epilogue<EPI>(row, sum, y, e, s, a0, a1);
        __syncthreads();   // stage sidx is free again
        if (tid == 0 && !failed) {
            const int tn = t + 2 * G;
            if (tn < ntiles) tile_issue<CAP>(__ldg(tiles + tn), st + sidx, bar + sidx, rowptr, colidx, vals);
        }
    }
    if (failed && tid == 0) {
        // give the copies still in flight a bounded chance to land before the block exits
        for (int j = 0; j < 2; ++j) mbar_wait_bounded(bar + j, 0u);
    }
    if (EPI != EPI_NONE || f.kind != FIN_NONE) reduce_and_finish(a0, a1, ctl, partials, f);
}

cudaError_t spmv_tiled_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define TACTA_TILED_ATTR(CAP, EPI)                                                                   \
    if (e == cudaSuccess)                                                                            \
        e = cudaFuncSetAttribute(spmv_tiled<CAP, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 (int)spmv_tiled_smem(CAP));
    TACTA_TILED_ATTR(kTileCapSmall, EPI_NONE) TACTA_TILED_ATTR(kTileCapSmall, EPI_NORM)
    TACTA_TILED_ATTR(kTileCapSmall, EPI_RESID) TACTA_TILED_ATTR(kTileCapSmall, EPI_TAPIVOT)
    TACTA_TILED_ATTR(kTileCapLarge, EPI_NONE) TACTA_TILED_ATTR(kTileCapLarge, EPI_NORM)
    TACTA_TILED_ATTR(kTileCapLarge, EPI_RESID) TACTA_TILED_ATTR(kTileCapLarge, EPI_TAPIVOT)
#undef TACTA_TILED_ATTR
    if (e == cudaSuccess) done = true;
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

template <class Acc>
static cudaError_t spmv_dispatch(const LaunchCtx& L, int kind, const Acc& acc, const double* x,
                                 double* y, int epi, EpiArgs e, FinArgs f, int gate) {
    switch (epi) {
    case EPI_NONE: return spmv_dispatch_epi<Acc, EPI_NONE>(L, kind, acc, x, y, e, f, gate);
    case EPI_NORM: return spmv_dispatch_epi<Acc, EPI_NORM>(L, kind, acc, x, y, e, f, gate);
    case EPI_RESID: return spmv_dispatch_epi<Acc, EPI_RESID>(L, kind, acc, x, y, e, f, gate);
    default: return spmv_dispatch_epi<Acc, EPI_TAPIVOT>(L, kind, acc, x, y, e, f, gate);
    }
}

cudaError_t launch_spmv(const LaunchCtx& L, const DevOperand& A, const double* x, double* y,
                        int epi, EpiArgs e, FinArgs f, int gate) {
    if (A.format == TACTA_CSR && A.csr.cfg.kind == 2) {
        switch (epi) {
        case EPI_NONE: return spmv_tiled_launch<EPI_NONE>(L, A.csr, x, y, e, f, gate);
        case EPI_NORM: return spmv_tiled_launch<EPI_NORM>(L, A.csr, x, y, e, f, gate);
        case EPI_RESID: return spmv_tiled_launch<EPI_RESID>(L, A.csr, x, y, e, f, gate);
        default: return spmv_tiled_launch<EPI_TAPIVOT>(L, A.csr, x, y, e, f, gate);
        }
    }
    if (A.format == TACTA_CSR) {
        CsrAcc acc{A.csr.rowptr, A.csr.colidx, A.csr.vals, A.csr.rows};
        return spmv_dispatch(L, A.csr.cfg.kind, acc, x, y, epi, e, f, gate);
    }
    DenseAcc acc{A.dense.vals, A.dense.rows, A.dense.cols};
    return spmv_dispatch(L, A.dense.cfg.kind, acc, x, y, epi, e, f, gate);
}

// ------------------------------------------------------------------ vector kernels

struct VecPtrs { double* p[kTMax]; };

// CTA update (Eqs. CTAGEN7, CTAGEN7A): x += sum alpha_i z_i, r -= sum alpha_i u_i, ||r||².
template <int T>
__global__ void __launch_bounds__(kBlock)
cta_update(int64_t m, int64_t n, double* __restrict__ x, double* __restrict__ r, VecPtrs z,
           VecPtrs u, Ctl* ctl, double* partials, FinArgs f) {
    if (ctl->status != 0) return;
    double al[T];
#pragma unroll
    for (int j = 0; j < T; ++j) al[j] = ctl->alpha[j];
    double a0 = 0.0;
    const int64_t len = m > n ? m : n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
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
    reduce_and_finish(a0, 0.0, ctl, partials, f);
}

// TA update (Alg. 2.2): d = (1-alpha) d + alpha (b - v)  [d = b - b'],
// x = (1-alpha) x + (alpha s) c; reductions ||d||², dᵀb for the next iteration.
__global__ void __launch_bounds__(kBlock)
ta_update(int64_t m, int64_t n, double* __restrict__ x, double* __restrict__ d,
          const double* __restrict__ b, const double* __restrict__ v, const double* __restrict__ c,
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
            const double dv = om * d[i] + al * (bv - __ldg(v + i));
            d[i] = dv;
            a0 = fma(dv, dv, a0);
            a1 = fma(dv, bv, a1);
        }
        if (i < n) x[i] = om * x[i] + as * __ldg(c + i);
    }
    reduce_and_finish(a0, a1, ctl, partials, f);
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

cudaError_t launch_fill(const LaunchCtx& L, double* dst, double v, int64_t len) {
    fill_kernel<<<L.max_grid, kBlock, 0, L.stream>>>(dst, v, len);
    if (L.launches) ++*L.launches;
    return cudaGetLastError();
}

}  // namespace tacta
