// Solve of CTA's auxiliary equation, shared by the single-system and batched paths.
#pragma once

#include <cmath>

#include "internal.h"

// Round-to-nearest FP64 operations without contraction, on the device and on the host
// (the host build of this file compiles with -ffp-contract=off).
#ifdef __CUDA_ARCH__
#define TACTA_MUL(a, b) __dmul_rn((a), (b))
#define TACTA_SUB(a, b) __dsub_rn((a), (b))
#define TACTA_DIV(a, b) __ddiv_rn((a), (b))
#define TACTA_SQRT(a) __dsqrt_rn(a)
#else
#define TACTA_MUL(a, b) ((a) * (b))
#define TACTA_SUB(a, b) ((a) - (b))
#define TACTA_DIV(a, b) ((a) / (b))
#define TACTA_SQRT(a) std::sqrt(a)
#endif

namespace tacta {

// Auxiliary equation of order t (Eq. eqcoeff): [phi_{i+j}] alpha = [phi_i].
// Jacobi scaling G = D [phi_{i+j}] D, D = diag(phi_{2i})^{-1/2}, then the
// square-root-free Cholesky factorisation G = L diag(d) Lᵀ (L unit lower) in
// natural order, truncated at the first pivot d_k <= pivot_tol (d_k is the square
// of the k-th Cholesky pivot, so the truncation is the Cholesky one); the leading
// block is solved and the trailing alphas are 0.
// This runs on one thread while the rest of the device waits, so it is written for
// latency: the order is a template parameter (every loop unrolls and every array
// lives in registers, not local memory), the moments are loaded up front, and
// there is one division per pivot (FP64 division and square root are long
// dependent chains on this GPU).
template <int T>
static __host__ __device__ __forceinline__ int hankel_solve_t(const double* phi_in, double pivot_tol, double* alpha) {
    double phi[2 * T + 1];
#pragma unroll
    for (int i = 1; i <= 2 * T; ++i) phi[i] = phi_in[i];
    int tt = T;
#pragma unroll
    for (int i = T; i >= 1; --i)
        if (!(phi[2 * i] > 0.0)) tt = i - 1;
    double s[T], L[T][T], d[T], dinv[T], y[T], beta[T];
#pragma unroll
    for (int i = 0; i < T; ++i) s[i] = i < tt ? TACTA_DIV(1.0, TACTA_SQRT(phi[2 * i + 2])) : 0.0;
    int rank = 0;
    bool go = true;
#pragma unroll
    for (int k = 0; k < T; ++k) {
        if (go && k < tt) {
            double dk = TACTA_MUL(TACTA_MUL(s[k], phi[2 * k + 2]), s[k]);
#pragma unroll
            for (int j = 0; j < k; ++j) dk = TACTA_SUB(dk, TACTA_MUL(TACTA_MUL(L[k][j], L[k][j]), d[j]));
            if (dk > pivot_tol) {
                d[k] = dk;
                dinv[k] = TACTA_DIV(1.0, dk);
#pragma unroll
                for (int i = k + 1; i < T; ++i) {
                    double v = TACTA_MUL(TACTA_MUL(s[i], phi[i + k + 2]), s[k]);
#pragma unroll
                    for (int j = 0; j < k; ++j) v = TACTA_SUB(v, TACTA_MUL(TACTA_MUL(L[i][j], L[k][j]), d[j]));
                    L[i][k] = TACTA_MUL(v, dinv[k]);
                }
                rank = k + 1;
            } else {
                go = false;
            }
        }
    }
    double w[T];
#pragma unroll
    for (int i = 0; i < T; ++i) {               // L w = D phi_{1..}
        double v = TACTA_MUL(s[i], phi[i + 1]);
#pragma unroll
        for (int j = 0; j < i; ++j) v = TACTA_SUB(v, TACTA_MUL(L[i][j], w[j]));
        w[i] = i < rank ? v : 0.0;
    }
#pragma unroll
    for (int i = 0; i < T; ++i) y[i] = i < rank ? TACTA_MUL(w[i], dinv[i]) : 0.0;   // y = diag(d)^{-1} w
#pragma unroll
    for (int i = T - 1; i >= 0; --i) {          // Lᵀ beta = diag(d)^{-1} y
        double v = y[i];
#pragma unroll
        for (int j = i + 1; j < T; ++j)
            if (j < rank) v = TACTA_SUB(v, TACTA_MUL(L[j][i], beta[j]));
        beta[i] = v;
    }
#pragma unroll
    for (int i = 0; i < T; ++i) alpha[i] = i < rank ? TACTA_MUL(s[i], beta[i]) : 0.0;
    return rank;
}

static __host__ __device__ __noinline__ int hankel_solve_dev(const double* phi, int t, double pivot_tol, double* alpha) {
    switch (t) {
    case 1: return hankel_solve_t<1>(phi, pivot_tol, alpha);
    case 2: return hankel_solve_t<2>(phi, pivot_tol, alpha);
    case 3: return hankel_solve_t<3>(phi, pivot_tol, alpha);
    case 4: return hankel_solve_t<4>(phi, pivot_tol, alpha);
    case 5: return hankel_solve_t<5>(phi, pivot_tol, alpha);
    case 6: return hankel_solve_t<6>(phi, pivot_tol, alpha);
    case 7: return hankel_solve_t<7>(phi, pivot_tol, alpha);
    default: return hankel_solve_t<8>(phi, pivot_tol, alpha);
    }
}

}  // namespace tacta

#ifdef __CUDACC__
namespace tacta {

// The same solve by one warp, lane i holding row i of L: every value is formed by the same
// operations in the same order as hankel_solve_t<T> (so alpha is bit for bit the same),
// but the rows of each Cholesky column are computed in parallel and each lane keeps only
// its own row, which keeps the solve in registers inside kernels with a tight register
// budget. Every lane of the warp must call it; lanes i < T write alpha[i]; returns the
// rank (the same in every lane).
template <int T>
__device__ __forceinline__ int hankel_solve_warp_t(const double* phi, double pivot_tol, double* alpha) {
    const int i = threadIdx.x & 31;
    int tt = T;
#pragma unroll
    for (int k = T; k >= 1; --k)
        if (!(phi[2 * k] > 0.0)) tt = k - 1;
    const double si = i < tt ? TACTA_DIV(1.0, TACTA_SQRT(phi[2 * i + 2])) : 0.0;
    double Lr[T], d[T];
    double my_dinv = 0.0;
#pragma unroll
    for (int j = 0; j < T; ++j) { Lr[j] = 0.0; d[j] = 0.0; }
    int rank = 0;
    bool go = true;
#pragma unroll
    for (int k = 0; k < T; ++k) {
        if (go && k < tt) {
            const double sk = __shfl_sync(0xffffffffu, si, k);
            double dk = TACTA_MUL(TACTA_MUL(sk, phi[2 * k + 2]), sk);
#pragma unroll
            for (int j = 0; j < k; ++j) {
                const double lkj = __shfl_sync(0xffffffffu, Lr[j], k);
                dk = TACTA_SUB(dk, TACTA_MUL(TACTA_MUL(lkj, lkj), d[j]));
            }
            if (dk > pivot_tol) {
                d[k] = dk;
                const double dinv = TACTA_DIV(1.0, dk);
                if (i == k) my_dinv = dinv;
                double v = TACTA_MUL(TACTA_MUL(si, phi[(i < T ? i : 0) + k + 2]), sk);
#pragma unroll
                for (int j = 0; j < k; ++j) {
                    const double lkj = __shfl_sync(0xffffffffu, Lr[j], k);
                    v = TACTA_SUB(v, TACTA_MUL(TACTA_MUL(Lr[j], lkj), d[j]));
                }
                if (i > k && i < T) Lr[k] = TACTA_MUL(v, dinv);
                rank = k + 1;
            } else {
                go = false;
            }
        }
    }
    // L w = D phi_{1..}: lane i subtracts L[i][j] w_j as w_j becomes known (j ascending,
    // the order of the row sum in hankel_solve_t)
    double v = i < T ? TACTA_MUL(si, phi[i + 1]) : 0.0;
    double wmine = 0.0;
#pragma unroll
    for (int j = 0; j < T; ++j) {
        double wj = __shfl_sync(0xffffffffu, v, j);
        wj = j < rank ? wj : 0.0;
        if (i == j) wmine = wj;
        if (i > j) v = TACTA_SUB(v, TACTA_MUL(Lr[j], wj));
    }
    const double yi = i < rank ? TACTA_MUL(wmine, my_dinv) : 0.0;
    // column i of L into lane i (Lc[j] = L[j][i], j > i)
    double Lc[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
        Lc[j] = 0.0;
#pragma unroll
        for (int c = 0; c < j; ++c) {
            const double ljc = __shfl_sync(0xffffffffu, Lr[c], j);
            if (i == c) Lc[j] = ljc;
        }
    }
    // Lᵀ beta = y, rows from the last: lane i's sum runs over j = i+1.. ascending
    double beta_mine = 0.0;
    double bj[T];
#pragma unroll
    for (int k = T - 1; k >= 0; --k) {
        double b = yi;
#pragma unroll
        for (int j = k + 1; j < T; ++j)
            if (j < rank) b = TACTA_SUB(b, TACTA_MUL(Lc[j], bj[j]));
        bj[k] = __shfl_sync(0xffffffffu, b, k);
        if (i == k) beta_mine = b;
    }
    if (i < T) alpha[i] = i < rank ? TACTA_MUL(si, beta_mine) : 0.0;
    return rank;
}

static __device__ __noinline__ int hankel_solve_warp(const double* phi, int t, double pivot_tol, double* alpha) {
    switch (t) {
    case 1: return hankel_solve_warp_t<1>(phi, pivot_tol, alpha);
    case 2: return hankel_solve_warp_t<2>(phi, pivot_tol, alpha);
    case 3: return hankel_solve_warp_t<3>(phi, pivot_tol, alpha);
    case 4: return hankel_solve_warp_t<4>(phi, pivot_tol, alpha);
    case 5: return hankel_solve_warp_t<5>(phi, pivot_tol, alpha);
    case 6: return hankel_solve_warp_t<6>(phi, pivot_tol, alpha);
    case 7: return hankel_solve_warp_t<7>(phi, pivot_tol, alpha);
    default: return hankel_solve_warp_t<8>(phi, pivot_tol, alpha);
    }
}

}  // namespace tacta
#endif
