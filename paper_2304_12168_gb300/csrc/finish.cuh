// Device-side control logic shared by the streaming kernels (kernels.cu) and the fused
// cooperative kernels (chain.cu): gates, the one-thread finishers that take the stop,
// pivot and step decisions of Alg. 1.1 / 2.1 / 2.2, and the deterministic block and
// grid reductions that feed them.
#pragma once

#include <cfloat>
#include <cstdint>

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
static __device__ void loop_top(Ctl* c) {
    if (!finite(c->rn2)) { c->status = TACTA_REASON_NONFINITE; return; }
    if (c->rn2 <= c->res_thr) {
        if (c->is_true) { c->status = TACTA_REASON_RESIDUAL; return; }
        c->need_true = 1;
        return;
    }
    if (c->k >= c->max_iter) c->status = TACTA_REASON_MAXITER;
}

// the history holds ||r||² / ||b||² while the solve runs (a multiply: FP64 division and
// square root are long dependent chains, and finishers run on one thread while the
// device waits); hist_sqrt turns it into ||r|| / ||b|| once, when it is copied out
static __device__ void put_hist(Ctl* c, double* h) {
    if (h != nullptr && c->k < c->hist_cap) {
        h[c->k] = __dmul_rn(c->rn2, c->inv_bn2);
        if (c->k + 1 > c->hist_len) c->hist_len = c->k + 1;
    }
}

static __device__ __noinline__ void finish(Ctl* c, const FinArgs& f, double r0, double r1) {
    if (c->status == TACTA_REASON_TIMEOUT) return;   // a kernel gave up waiting: keep that verdict
    switch (f.kind) {
    case FIN_STORE:
        c->red[f.idx] = r0;
        c->red[f.idx + 1] = r1;
        break;
    case FIN_PHI:
        c->phi[f.idx] = r0;
        break;
    case FIN_CTA_UPDATE:
        c->k += 1;
        c->is_true = 0;
        c->rn2 = r0;
        put_hist(c, f.hist);
        if (c->enh_stop) { c->status = TACTA_REASON_ENHANCED; break; }
        if (c->R > 0 && c->k % c->R == 0) { c->need_true = 1; break; }
        if (c->ref_eta2 > 0.0 && r0 <= c->ref_thr) { c->need_true = 1; break; }
        loop_top(c);
        break;
    case FIN_TRUE_RES:
        c->rn2 = r0;
        c->db = r1;
        c->is_true = 1;
        c->need_true = 0;
        c->ref_thr = __dmul_rn(c->ref_eta2, r0);
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
        if (c->nonneg) {
            // c_+ ~ 0 with (b - b')ᵀb > 0: Farkas certificate of infeasibility (Sec. 6 reading)
            if (r0 <= c->nrm_thr && c->db > 0.0) { c->status = TACTA_REASON_WITNESS; return; }
        } else if (r0 <= c->nrm_thr) {
            c->status = TACTA_REASON_NORMAL;
            return;
        }
        const double cn = __dsqrt_rn(r0);
        if (__dmul_rn(c->rho, cn) >= c->db) {            // strict pivot (Eq. eqlem2)
            c->pivot = 1;
            c->s = cn > 0.0 ? __ddiv_rn(c->rho, cn) : 0.0;   // c_+ = 0: the pivot is v = 0
        } else {
            c->pivot = 0;
            if (c->grow_rho) {
                c->rho = fmax(__dmul_rn(2.0, c->rho), __ddiv_rn(c->db, cn));
                if (c->rho > c->rho_max) c->status = TACTA_REASON_RHO_BOUND;
            } else {
                c->status = TACTA_REASON_WITNESS;      // Alg. 2.1 STOP
            }
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
        c->inv_bn2 = r0 > 0.0 ? __ddiv_rn(1.0, r0) : 0.0;
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

// Sum of one value over a block of kBlock threads, result valid in warp 0.
// An FP64 warp-instruction costs the same on GB300 whatever the number of
// active lanes, so the values go through shared memory and warp 0 alone adds
// them (7 + 5 FP64 warp-instructions, instead of a shuffle tree in every warp).
template <int NT = kBlock>
__device__ __forceinline__ double block_sum_warp0(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = sh[threadIdx.x];
#pragma unroll
        for (int i = 1; i < NT / 32; ++i) s += sh[threadIdx.x + 32 * i];
        s = warp_sum(s);
    }
    __syncthreads();
    return s;
}

// Block-level reduction of NRED values (a0 and, if NRED = 2, a1), one partial
// per block; the last block to finish (atomic ticket, no waiting) sums the
// partials in block order and runs the finisher. Requires blockDim = NT.
// STAGED: the finisher runs against a shared-memory copy of the control block, loaded and
// stored by the block's threads at once (for the vector kernels, whose finishers read and
// write a dozen fields); otherwise it works on the control block in global memory.
template <int NRED = 2, int NT = kBlock, bool STAGED = false>
__device__ void reduce_and_finish(double a0, double a1, Ctl* ctl, double* partials,
                                  const FinArgs& f) {
    __shared__ double sh[NT];
    __shared__ int am_last;
    const double s0 = block_sum_warp0<NT>(a0, sh);
    const double s1 = NRED > 1 ? block_sum_warp0<NT>(a1, sh) : 0.0;
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = s0;
        partials[2 * blockIdx.x + 1] = s1;
        __threadfence();
        const unsigned ticket = atomicAdd(&ctl->counter, 1u);
        am_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    if constexpr (STAGED) {
        __shared__ Ctl sc;
        constexpr int kWords = (int)(sizeof(Ctl) / 8);
        static_assert(sizeof(Ctl) % 8 == 0 && kWords <= NT, "the control block copies as one word per thread");
        uint64_t* cw = reinterpret_cast<uint64_t*>(ctl);
        uint64_t* sw = reinterpret_cast<uint64_t*>(&sc);
        if (threadIdx.x < kWords) sw[threadIdx.x] = __ldcg(cw + threadIdx.x);
        double t0 = 0.0, t1 = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            t0 += __ldcg(&partials[2 * i]);
            if (NRED > 1) t1 += __ldcg(&partials[2 * i + 1]);
        }
        t0 = block_sum_warp0<NT>(t0, sh);   // its barriers also publish the staged copy
        if (NRED > 1) t1 = block_sum_warp0<NT>(t1, sh);
        if (threadIdx.x == 0) {
            sc.counter = 0;
            if (f.reset_bar) sc.chain_bar = 0;   // every block of a fused step is past its grid waits
            finish(&sc, f, t0, t1);
        }
        __syncthreads();
        if (threadIdx.x < kWords) cw[threadIdx.x] = sw[threadIdx.x];
    } else {
        double t0 = 0.0, t1 = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            t0 += __ldcg(&partials[2 * i]);
            if (NRED > 1) t1 += __ldcg(&partials[2 * i + 1]);
        }
        t0 = block_sum_warp0<NT>(t0, sh);
        if (NRED > 1) t1 = block_sum_warp0<NT>(t1, sh);
        if (threadIdx.x == 0) {
            ctl->counter = 0;
            if (f.reset_bar) ctl->chain_bar = 0;
            finish(ctl, f, t0, t1);
        }
    }
}

}  // namespace tacta
