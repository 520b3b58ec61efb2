"""Centering Triangle Algorithm (CTA), oracle form (test infrastructure only).

Follows Sec. 3 of Lau & Kalantari (arXiv:2304.12168) with H = A Aᵀ, the choice
the paper's implementation always makes (Sec. 5, "we always use H = AAᵀ").

One iteration of order t (Eqs. F_t, eqcoeff, CTAGEN7, CTAGEN7A):

    phi_i = rᵀ H^i r,  i = 1..2t
    solve the t x t auxiliary (Hankel) system  [phi_{i+j}] alpha = [phi_i]
    r'' = r' - sum_i alpha_i H^i r'
    x'' = x' + sum_i alpha_i Aᵀ H^{i-1} r'

With H = A Aᵀ the moments are norms of the chain u_0 = r, z_i = Aᵀ u_{i-1},
u_i = A z_i:  H^i r = u_i,  Aᵀ H^{i-1} r = z_i,  phi_{2i-1} = ||z_i||²,
phi_{2i} = ||u_i||².

Readings where the paper leaves a choice open (each one is shared by the CUDA
solver):
  * t-cycling (Sec. 5.1): "ping-pong" 1,2,3,4,5,4,3,2,1,2,... -- after F_5 the
    next step is F_4, as the paper's example says; one iteration = one F_t.
  * stopping (Alg. 1.1 while-clauses): relative forms ||r|| <= tol ||b|| and
    ||Aᵀ r|| <= tol_normal ||Aᵀ b|| (the paper's second clause rᵀ H r is the
    square of ||Aᵀ r||).
  * residual: r is updated recursively (Eq. CTAGEN7); every R iterations, and
    whenever the recursive r passes the residual test, r is replaced by the
    true b - A x and the test is taken on that.
  * auxiliary solve: the paper asks for the minimum-norm solution when the
    Hankel matrix is singular. The step (x'', r'') is the same for every
    least-squares solution (every z_i lies in range(Aᵀ), on which A is
    one-to-one), so the oracle solves the leading nonsingular block:
    Jacobi scaling D = diag(G)^(-1/2), Cholesky of D G D in natural order,
    stopping at the first pivot <= pivot_tol; the trailing alphas are 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .status import Status, Reason

PINGPONG, SAWTOOTH, FIXED = 0, 1, 2


def schedule(k: int, t_max: int, cycle: int = PINGPONG) -> int:
    """Order t of iteration k (k = 0, 1, 2, ...), Sec. 5.1 t-cycling.

    PINGPONG with t_max = 5 gives 1,2,3,4,5,4,3,2, 1,2,3,... ;
    SAWTOOTH gives 1..t_max, 1..t_max, ... ; FIXED always gives t_max.
    """
    if cycle == FIXED or t_max == 1:
        return t_max
    if cycle == SAWTOOTH:
        return 1 + k % t_max
    period = 2 * t_max - 2
    j = k % period
    return j + 1 if j < t_max else 2 * t_max - 1 - j


def hankel_solve(phi, t: int, pivot_tol: float = 1e-12):
    """Solve the auxiliary equation (Eq. eqcoeff) of order t.

    phi is indexable as phi[1] .. phi[2t] (phi[0] is ignored). Returns
    (alpha[0..t-1], rank) where rank is the size of the leading block that was
    solved; alpha[rank:] = 0. rank = 0 means phi_2 = 0 (H r = 0).
    """
    # Jacobi scaling s_i = phi_{2i}^(-1/2); a non-positive diagonal ends the block
    tt = 0
    s = []
    for i in range(1, t + 1):
        if not phi[2 * i] > 0.0:
            break
        s.append(1.0 / math.sqrt(phi[2 * i]))
        tt = i
    # scaled Hankel matrix  Gs[i][j] = s_i phi_{i+j} s_j  (0-based i, j)
    Gs = [[s[i] * phi[i + j + 2] * s[j] for j in range(tt)] for i in range(tt)]
    L = [[0.0] * tt for _ in range(tt)]
    rank = 0
    for k in range(tt):
        d = Gs[k][k]
        for j in range(k):
            d -= L[k][j] * L[k][j]
        if not d > pivot_tol:
            break
        L[k][k] = math.sqrt(d)
        for i in range(k + 1, tt):
            v = Gs[i][k]
            for j in range(k):
                v -= L[i][j] * L[k][j]
            L[i][k] = v / L[k][k]
        rank = k + 1
    # forward / back substitution on the leading rank x rank block
    g = [s[i] * phi[i + 1] for i in range(rank)]
    y = [0.0] * rank
    for i in range(rank):
        v = g[i]
        for j in range(i):
            v -= L[i][j] * y[j]
        y[i] = v / L[i][i]
    beta = [0.0] * rank
    for i in reversed(range(rank)):
        v = y[i]
        for j in range(i + 1, rank):
            v -= L[j][i] * beta[j]
        beta[i] = v / L[i][i]
    alpha = [0.0] * t
    for i in range(rank):
        alpha[i] = s[i] * beta[i]
    return alpha, rank


def cta_chain(A, r, t: int):
    """The product chain of one F_t step with H = A Aᵀ.

    Returns (z[1..t], u[1..t], phi[0..2t]) with z_i = Aᵀ u_{i-1}, u_i = A z_i,
    u_0 = r, phi_{2i-1} = ||z_i||², phi_{2i} = ||u_i||² (phi[0] unused).
    """
    z, u = [], []
    phi = [0.0] * (2 * t + 1)
    prev = r
    for i in range(1, t + 1):
        zi = A.rmatvec(prev)
        phi[2 * i - 1] = float(zi @ zi)
        ui = A.matvec(zi)
        phi[2 * i] = float(ui @ ui)
        z.append(zi)
        u.append(ui)
        prev = ui
    return z, u, phi


def cta_step(A, x, r, t: int, pivot_tol: float = 1e-12):
    """One application of F_t (Eqs. CTAGEN7, CTAGEN7A) from (x', r').

    Returns (x'', r'', alpha, rank, phi).
    """
    z, u, phi = cta_chain(A, r, t)
    alpha, rank = hankel_solve(phi, t, pivot_tol)
    x2 = x.copy()
    r2 = r.copy()
    for i in range(t):
        x2 += alpha[i] * z[i]
        r2 -= alpha[i] * u[i]
    return x2, r2, alpha, rank, phi


def enhanced_stop(A, x, r, jmax: int, thr: float):
    """The enhanced stop of Sec. 3.2 from (x', r'): apply the first-order map
    F_1(r) = r - alpha_{1,1}(r) H r, alpha_{1,1}(r) = rᵀHr / rᵀH²r, j = 1, 2, ... times and
    return (x^, r_j, j) for the smallest j <= jmax with r_jᵀ H r_j <= thr, where
    x^ = x' + sum_{i<j} alpha_{1,1}(r_i) Aᵀ r_i (Eq. widehatxB, H = A Aᵀ); None if no j does.
    """
    xh = np.array(x, dtype=np.float64)
    ri = np.array(r, dtype=np.float64)
    for j in range(1, jmax + 1):
        w = A.rmatvec(ri)                 # Aᵀ r_{j-1}
        hr = A.matvec(w)                  # H r_{j-1}
        den = float(hr @ hr)
        if not den > 0.0:
            return None
        a = float(w @ w) / den            # alpha_{1,1}(r_{j-1})
        xh = xh + a * w
        ri = ri - a * hr
        wj = A.rmatvec(ri)
        if float(wj @ wj) <= thr:         # r_jᵀ H r_j = ||Aᵀ r_j||²
            return xh, ri, j
    return None


@dataclass
class CTAResult:
    x: np.ndarray
    status: Status
    reason: Reason
    iters: int
    matvecs: int
    hist: list = field(default_factory=list)
    rel_res: float = float("nan")          # true ||b - A x|| / ||b|| at exit
    rel_normal_res: float = float("nan")   # true ||Aᵀ(b - A x)|| / ||Aᵀ b|| at exit
    r: np.ndarray | None = None            # the residual the iteration carried at exit


def cta_solve(A, b, x0=None, tol=1e-10, tol_normal=None, max_iter=1000, t_max=5,
              cycle=PINGPONG, recompute_every=40, pivot_tol=1e-12, observer=None,
              enhanced=False) -> CTAResult:
    """Algorithm 1.1 (CTA) with H = A Aᵀ and the Sec. 5.1 t-cycling.

    Loop (k counts completed F_t steps; hist[k] = ||r_k|| / ||b||):
      1. if ||r|| <= tol ||b||: if r is the recursive residual, replace it by the
         true b - A x (and hist[k] by its norm); stop if it still passes.
      2. stop if k = max_iter.
      3. t = t(k); chain z_i, u_i and moments phi_1..phi_2t.
      4. stop if phi_1 = ||Aᵀ r||² <= tol_normal² ||Aᵀ b||² (normal equation
         solved, Alg. 1.1 second clause); with ``enhanced`` and t >= 2, the enhanced
         algorithm of Sec. 3.2 also stops here when a first-order iterate F_1^j(r),
         j <= t - 1, meets that test, with x = x^ of Eq. widehatxB (counted as a step).
      5. alpha from the auxiliary equation; rank 0 -> breakdown.
      6. x += sum alpha_i z_i, r -= sum alpha_i u_i; k += 1; every R-th k the
         true residual replaces r.

    ``observer(k, x, r, t, alpha, rank, phi)``, if given, is called after every
    completed step (used by the invariant tests).
    """
    if tol_normal is None:
        tol_normal = tol
    m, n = A.m, A.n
    b = np.asarray(b, dtype=np.float64)
    start = A.nmatvec
    bn2 = float(b @ b)
    if bn2 == 0.0:
        x = np.zeros(n)
        return CTAResult(x, Status.OK, Reason.ZERO_RHS, 0, 0, [0.0], 0.0, 0.0, np.zeros(m))
    atb = A.rmatvec(b)
    atbn2 = float(atb @ atb)
    res_thr = tol * tol * bn2
    nrm_thr = tol_normal * tol_normal * atbn2
    if x0 is None:
        x = np.zeros(n)
        r = b.copy()
    else:
        x = np.array(x0, dtype=np.float64)
        r = b - A.matvec(x)
    is_true = True
    rn2 = float(r @ r)
    hist = [math.sqrt(rn2 / bn2)]
    k = 0
    status, reason = Status.MAXITER, Reason.MAXITER
    while True:
        if not math.isfinite(rn2):
            status, reason = Status.NONFINITE, Reason.NONFINITE
            break
        if rn2 <= res_thr:
            if not is_true:
                r = b - A.matvec(x)
                is_true = True
                rn2 = float(r @ r)
                hist[k] = math.sqrt(rn2 / bn2)
            if rn2 <= res_thr:
                status, reason = Status.OK, Reason.RESIDUAL
                break
        if k >= max_iter:
            status, reason = Status.MAXITER, Reason.MAXITER
            break
        t = schedule(k, t_max, cycle)
        z, u, phi = cta_chain(A, r, t)
        if not all(math.isfinite(p) for p in phi[1:]):
            status, reason = Status.NONFINITE, Reason.NONFINITE
            break
        if phi[1] <= nrm_thr:
            status, reason = Status.OK, Reason.NORMAL
            break
        if enhanced and t >= 2:
            hit = enhanced_stop(A, x, r, t - 1, nrm_thr)
            if hit is not None:
                x, r, _ = hit
                k += 1
                is_true = False
                rn2 = float(r @ r)
                hist.append(math.sqrt(rn2 / bn2))
                status, reason = Status.OK, Reason.ENHANCED
                break
        alpha, rank = hankel_solve(phi, t, pivot_tol)
        if rank == 0:
            status, reason = Status.BREAKDOWN, Reason.BREAKDOWN
            break
        for i in range(t):
            x += alpha[i] * z[i]
            r -= alpha[i] * u[i]
        k += 1
        is_true = False
        if recompute_every and k % recompute_every == 0:
            r = b - A.matvec(x)
            is_true = True
        if observer is not None:
            observer(k, x, r, t, alpha, rank, phi)
        rn2 = float(r @ r)
        hist.append(math.sqrt(rn2 / bn2))
    matvecs = A.nmatvec - start
    rt = b - A.matvec(x)
    nrt = A.rmatvec(rt)
    rel_res = math.sqrt(float(rt @ rt) / bn2)
    rel_nrm = math.sqrt(float(nrt @ nrt) / atbn2) if atbn2 > 0 else 0.0
    return CTAResult(x, status, reason, k, matvecs, hist, rel_res, rel_nrm, r)
