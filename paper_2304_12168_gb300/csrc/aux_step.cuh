// The CTA step decision of Alg. 1.1 (Eq. eqcoeff) taken on the device after a step's
// chain of products: the moments summed from per-block partials, the normal-equation
// and finiteness tests, the enhanced stop of Sec. 3.2 and the auxiliary (Hankel) solve.
// Shared by the one-block cta_aux_step kernel (per-product chain) and the fused step
// kernel, where every block takes the decision redundantly from the same partials.
#pragma once

#include "finish.cuh"
#include "hankel.cuh"
#include "internal.h"

namespace tacta {

// Sum of G per-block partials by one warp: lanes stride over them with two accumulators,
// then a shuffle tree; the order depends on G only, so every block (of any size) that
// runs it gets the same bits. The result is valid in lane 0.
__device__ __forceinline__ double warp_sum_partials(const double* pw, int G) {
    const int lane = threadIdx.x & 31;
    double s0 = 0.0, s1 = 0.0;
    int i = lane;
#pragma unroll 4
    for (; i + 32 < G; i += 64) {
        s0 += __ldcg(pw + i);
        s1 += __ldcg(pw + i + 32);
    }
    if (i < G) s0 += __ldcg(pw + i);
    return warp_sum(s0 + s1);
}

// phi_{w+1} = sum over blocks of part[w * G + block], w = 0 .. 2t-1, into sc->phi (and
// into c->phi when c is not null), a warp per moment. rot shifts which warp takes which
// moment (an FP64 instruction holds its sub-partition's FP64 unit, so co-resident blocks
// spread their moment sums over different sub-partitions); the bits do not depend on it.
// Ends with __syncthreads().
__device__ __forceinline__ void sum_moment_partials(Ctl* sc, int t, const double* part, int G, Ctl* c,
                                                    int rot = 0) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int me = ((threadIdx.x >> 5) + nw - rot % nw) % nw;
    for (int w = me; w < 2 * t; w += nw) {
        const double s = warp_sum_partials(part + (size_t)w * G, G);
        if (lane == 0) {
            sc->phi[w + 1] = s;
            if (c) c->phi[w + 1] = s;
        }
    }
    __syncthreads();
}

// Enhanced stop (Sec. 3.2, Eq. widehatxB): the first-order iterates r_0 = r',
// r_{i+1} = r_i - a_i H r_i with a_i = r_iᵀH r_i / r_iᵀH² r_i are polynomials in H
// applied to r' (r_i = sum_k c_k H^k r'), so r_iᵀ H^s r_i = sum_{a,b} c_a c_b phi_{a+b+s}
// comes from the step's moments. If r_jᵀ H r_j <= thr for the smallest j <= t-1, the
// step's coefficients become those of x^ = x' + sum_{i<j} a_i Aᵀ r_i
// = x' + sum_k beta_k z_{k+1} (and r^ = r' - sum_k beta_k u_{k+1} = r_j), so the update
// applies x^ unchanged. Returns true if it stops there.
static __device__ __noinline__ bool enhanced_stop(Ctl* c, int t) {
    double cf[kTMax], beta[kTMax];
    for (int k = 0; k < kTMax; ++k) { cf[k] = 0.0; beta[k] = 0.0; }
    cf[0] = 1.0;
    for (int i = 0; i + 1 < t; ++i) {              // from r_i (degree i) to r_{i+1}
        double s1 = 0.0, s2 = 0.0;
        for (int a = 0; a <= i; ++a)
            for (int b = 0; b <= i; ++b) {
                const double w = __dmul_rn(cf[a], cf[b]);
                s1 = __fma_rn(w, c->phi[a + b + 1], s1);
                s2 = __fma_rn(w, c->phi[a + b + 2], s2);
            }
        if (!(s2 > 0.0)) return false;
        const double ai = __ddiv_rn(s1, s2);
        for (int k = 0; k <= i; ++k) beta[k] = __fma_rn(ai, cf[k], beta[k]);
        for (int k = i + 1; k >= 1; --k) cf[k] = __fma_rn(-ai, cf[k - 1], cf[k]);
        double q = 0.0;                              // r_{i+1}ᵀ H r_{i+1}
        for (int a = 0; a <= i + 1; ++a)
            for (int b = 0; b <= i + 1; ++b) q = __fma_rn(__dmul_rn(cf[a], cf[b]), c->phi[a + b + 1], q);
        if (q <= c->nrm_thr) {
            for (int k = 0; k < t; ++k) c->alpha[k] = beta[k];
            c->rank = i + 1;
            c->enh_stop = 1;
            return true;
        }
    }
    return false;
}

// One thread, on a copy sc of the control block holding the step's moments phi_1..phi_2t:
// finite moments, the normal-equation test (phi_1 = ||Aᵀ r||², scaled by cs2 on the FP32
// chain), the enhanced stop, then the auxiliary solve -> sc->alpha, sc->rank. Returns the
// stop reason (0: the step goes on to the update; it also goes on after an enhanced stop,
// with sc->enh_stop = 1, so the update applies x^).
static __device__ __forceinline__ int aux_decide(Ctl* sc, int t) {
    for (int i = 1; i <= 2 * t; ++i)
        if (!finite(sc->phi[i])) return TACTA_REASON_NONFINITE;
    if (sc->phi[1] <= __dmul_rn(sc->nrm_thr, sc->cs2)) return TACTA_REASON_NORMAL;
    if (sc->enhanced && t >= 2 && enhanced_stop(sc, t)) return 0;
    sc->rank = hankel_solve_dev(sc->phi, t, sc->pivot_tol, sc->alpha);
    return sc->rank == 0 ? TACTA_REASON_BREAKDOWN : 0;
}

}  // namespace tacta
