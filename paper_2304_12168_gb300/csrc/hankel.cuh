// Solve of CTA's auxiliary equation, shared by the single-system and batched paths.
#pragma once

#include "internal.h"

namespace tacta {

// Auxiliary equation of order t (Eq. eqcoeff): [phi_{i+j}] alpha = [phi_i].
// Jacobi-scaled Cholesky in natural order, truncated at the first pivot
// <= pivot_tol; the leading block is solved and the trailing alphas are 0.
// Arithmetic uses explicit round-to-nearest operations (no contraction).
static __device__ int hankel_solve_dev(const double* phi, int t, double pivot_tol, double* alpha) {
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

}  // namespace tacta
