"""Triangle Algorithm (TA), oracle form (test infrastructure only).

Follows Sec. 4 of Lau & Kalantari (arXiv:2304.12168):

  * ``ta_fixed_rho``  -- Algorithm 2.1: test b in E_{A,rho} = {Ax : ||x|| <= rho}.
  * ``ta_solve``      -- Algorithm 2.2: rho grows as max{2 rho, (b-b')ᵀb / ||c||}.
  * ``ta_minnorm_bisect`` -- Algorithm 2.5: bisection on rho between a lower
                         bound (Cor. cor1) and the norm of the best solution.
  * ``ta_minnorm``    -- the hybrid of Sec. 5.2: CTA to tol_cta first, then
                         Algorithm 2.5 on (A, b) if CTA's x solves A x = b,
                         else on (AᵀA, Aᵀb) through products only.

One TA iteration at iterate b' = A x' (Thm. prop0TA, Prop. prop1TA):

    c = Aᵀ (b - b')
    pivot test (Eq. eqlem2):  rho ||c|| >= (b - b')ᵀ b
    v = rho A c / ||c||                                  (Eq. vr)
    alpha = (b - b')ᵀ (v - b') / ||v - b'||²             (Eq. alph)
    b'' = (1 - alpha) b' + alpha v,  x'' = (1 - alpha) x' + alpha rho c / ||c||

Readings (shared with the CUDA solver):
  * stopping: ||b - b'|| <= tol ||b|| and ||c|| <= tol_normal ||Aᵀ b||
    (relative forms of the while-clauses). Alg. 2.5's inner clause
    ||Aᵀ(b - b')|| > 0 is read the same way.
  * alpha is clamped to at most 1 ("nearest point to b on the segment b'v";
    under the strict-pivot test alpha <= 1 already holds up to rounding).
  * b' is carried recursively; every R iterations, and when the recursive b'
    passes the residual test, it is replaced by A x'.
  * a warm start x0 sets b' = A x0 and rho = ||x0|| (keeps ||x'|| <= rho).
  * Alg. 2.5: rho is recomputed as the midpoint at the top of every outer
    trip; the gap test is rho_hi - rho_lo <= tol * ||x_eps||; each inner
    test starts from the last witness (x' = 0 before the first one).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .cta import cta_solve, PINGPONG
from .ops import NormalOperator
from .status import Status, Reason


@dataclass
class TAResult:
    x: np.ndarray
    bp: np.ndarray               # b' = A x' carried by the iteration
    status: Status
    reason: Reason
    iters: int
    matvecs: int
    rho: float
    hist: list = field(default_factory=list)
    db: float = float("nan")     # (b - b')ᵀ b at exit
    cn: float = float("nan")     # ||Aᵀ (b - b')|| at exit (when computed)
    rel_res: float = float("nan")
    rel_normal_res: float = float("nan")


def _ta_loop(M, b, x, bp, rho, grow_rho, tol, tol_normal, max_iter, recompute_every, mtb_n2,
             observer=None, nonneg=False, rho_max=math.inf):
    """The TA while-loop shared by Alg. 2.1 (grow_rho=False: a failed pivot
    test is a witness, STOP) and Alg. 2.2 (grow_rho=True: rho grows).

    nonneg=True is the LP-feasibility form of Sec. 6: c is replaced by
    c_+ = max(c, 0) (Eq. vrend2: the maximiser of c_+ᵀx over {Ax in E_{A,rho}, x >= 0}
    is rho c_+/||c_+||), so every iterate stays x' >= 0. Reading where the section is
    silent: when c_+ = 0 the maximiser is x = 0 (v = 0), still a strict pivot if
    (b-b')ᵀb <= 0; if ||c_+|| <= tol_normal ||Aᵀb|| and (b-b')ᵀb > 0 then d = b - b'
    certifies infeasibility up to that tolerance (Farkas: Aᵀd <= 0, bᵀd > 0) and the
    loop stops with WITNESS. The normal-equation stop does not apply; rho growing past
    rho_max (the section's termination bound) ends the loop with RHO_BOUND."""
    bn2 = float(b @ b)
    res_thr = tol * tol * bn2
    nrm_thr = tol_normal * tol_normal * mtb_n2
    is_true = True
    k = 0
    d = b - bp
    dn2 = float(d @ d)
    hist = [math.sqrt(dn2 / bn2)]
    db = cn = float("nan")
    status, reason = Status.MAXITER, Reason.MAXITER
    while True:
        if not math.isfinite(dn2):
            status, reason = Status.NONFINITE, Reason.NONFINITE
            break
        if dn2 <= res_thr:
            if not is_true:
                bp = M.matvec(x)
                is_true = True
                d = b - bp
                dn2 = float(d @ d)
                hist[k] = math.sqrt(dn2 / bn2)
            if dn2 <= res_thr:
                status, reason = Status.OK, Reason.RESIDUAL
                break
        if k >= max_iter:
            status, reason = Status.MAXITER, Reason.MAXITER
            break
        c = M.rmatvec(d)
        if nonneg:
            c = np.maximum(c, 0.0)
        cn2 = float(c @ c)
        db = float(d @ b)
        if not (math.isfinite(cn2) and math.isfinite(db)):
            status, reason = Status.NONFINITE, Reason.NONFINITE
            break
        cn = math.sqrt(cn2)
        if nonneg:
            # c_+ = 0 and (b-b')ᵀb > 0: d = b - b' has Aᵀd <= 0 and bᵀd > 0, a Farkas
            # certificate that A x = b, x >= 0 has no solution (a witness for every rho)
            if cn2 <= nrm_thr and db > 0.0:
                status, reason = Status.WITNESS, Reason.WITNESS
                break
        elif cn2 <= nrm_thr:
            status, reason = Status.OK, Reason.NORMAL
            break
        alpha = None
        if rho * cn >= db:
            # strict pivot v = rho A c / ||c|| (Thm. prop0TA) and step (Prop. prop1TA);
            # with c_+ = 0 the maximiser over {||x|| <= rho, x >= 0} is x = 0, so v = 0
            s = rho / cn if cn > 0.0 else 0.0
            v = s * M.matvec(c)
            w = v - bp
            num = float(d @ w)
            den = float(w @ w)
            if not den > 0.0:
                status, reason = Status.BREAKDOWN, Reason.BREAKDOWN
                break
            alpha = min(num / den, 1.0)
            bp = (1.0 - alpha) * bp + alpha * v
            x = (1.0 - alpha) * x + (alpha * s) * c
        elif grow_rho:
            rho = max(2.0 * rho, db / cn)          # Alg. 2.2 else-branch
            if rho > rho_max:
                status, reason = Status.OK, Reason.RHO_BOUND
                break
        else:
            status, reason = Status.WITNESS, Reason.WITNESS   # Alg. 2.1 STOP
            break
        k += 1
        is_true = False
        if recompute_every and k % recompute_every == 0:
            bp = M.matvec(x)
            is_true = True
        if observer is not None:
            observer(k, x, bp, rho, alpha)
        d = b - bp
        dn2 = float(d @ d)
        hist.append(math.sqrt(dn2 / bn2))
    return x, bp, rho, status, reason, k, hist, db, cn


def _finish(M, b, x, bp, status, reason, k, matvecs, rho, hist, db, cn, mtb_n2):
    bn2 = float(b @ b)
    rt = b - M.matvec(x)
    nrt = M.rmatvec(rt)
    return TAResult(x, bp, status, reason, k, matvecs, rho, hist, db, cn,
                    math.sqrt(float(rt @ rt) / bn2),
                    math.sqrt(float(nrt @ nrt) / mtb_n2) if mtb_n2 > 0 else 0.0)


def ta_solve(M, b, x0=None, tol=1e-10, tol_normal=None, max_iter=1000,
             recompute_every=40, observer=None, nonneg=False, rho_max=math.inf) -> TAResult:
    """Algorithm 2.2: rho = 0, x' = 0, b' = 0 (or the warm start x0).

    ``observer(k, x, b', rho, alpha)`` is called after every iteration
    (alpha is None on a rho-growth iteration). ``nonneg`` / ``rho_max``: the
    LP-feasibility form of Sec. 6 (see _ta_loop); a warm start must then be >= 0.
    """
    if tol_normal is None:
        tol_normal = tol
    b = np.asarray(b, dtype=np.float64)
    n = M.n
    if float(b @ b) == 0.0:
        z = np.zeros(n)
        return TAResult(z, np.zeros(M.m), Status.OK, Reason.ZERO_RHS, 0, 0, 0.0, [0.0],
                        rel_res=0.0, rel_normal_res=0.0)
    start = M.nmatvec
    mtb = M.rmatvec(b)
    mtb_n2 = float(mtb @ mtb)
    if x0 is None:
        x, bp, rho = np.zeros(n), np.zeros(M.m), 0.0
    else:
        x = np.array(x0, dtype=np.float64)
        bp = M.matvec(x)
        rho = float(np.linalg.norm(x))
    x, bp, rho, st, rs, k, hist, db, cn = _ta_loop(M, b, x, bp, rho, True, tol, tol_normal,
                                                   max_iter, recompute_every, mtb_n2, observer,
                                                   nonneg, rho_max)
    return _finish(M, b, x, bp, st, rs, k, M.nmatvec - start, rho, hist, db, cn, mtb_n2)


def ta_fixed_rho(M, b, rho, x_start=None, bp_start=None, tol=1e-10, tol_normal=None,
                 max_iter=1000, recompute_every=40, mtb_n2=None, observer=None) -> TAResult:
    """Algorithm 2.1 for a fixed rho, from (x_start, b'_start = A x_start) or 0.

    Ends with Status.OK (||b - b'|| <= tol ||b||, or ||c|| small: reason NORMAL),
    Status.WITNESS (pivot test failed; db / cn is a lower bound on ||x_*||,
    Cor. cor1) or Status.MAXITER.
    """
    if tol_normal is None:
        tol_normal = tol
    b = np.asarray(b, dtype=np.float64)
    start = M.nmatvec
    if mtb_n2 is None:
        mtb = M.rmatvec(b)
        mtb_n2 = float(mtb @ mtb)
    x = np.zeros(M.n) if x_start is None else np.array(x_start, dtype=np.float64)
    bp = np.zeros(M.m) if bp_start is None else np.array(bp_start, dtype=np.float64)
    x, bp, rho, st, rs, k, hist, db, cn = _ta_loop(M, b, x, bp, rho, False, tol, tol_normal,
                                                   max_iter, recompute_every, mtb_n2, observer)
    return TAResult(x, bp, st, rs, k, M.nmatvec - start, rho, hist, db, cn)


@dataclass
class MinNormResult:
    x: np.ndarray
    status: Status
    reason: Reason
    rho_upper: float
    rho_lower: float
    trips: int
    iters: int                  # TA iterations over all trips
    cta_iters: int = 0
    normal_system: bool = False
    trip_log: list = field(default_factory=list)   # (rho, status, rho_upper, rho_lower, iters)
    rel_res: float = float("nan")
    rel_normal_res: float = float("nan")


def ta_minnorm_bisect(M, b, x_eps, tol=1e-10, tol_normal=None, max_iter=10000,
                      recompute_every=40) -> MinNormResult:
    """Algorithm 2.5: given an approximate solution x_eps of M x = b, bisect on rho.

    rho_hi = ||x_eps||, rho_lo = 0; while rho_hi - rho_lo > tol ||x_eps||:
    rho = (rho_hi + rho_lo) / 2; run Alg. 2.1 at rho from the last witness;
    on success rho_hi = rho (that x is the new answer), on a witness
    rho_lo = (b - b')ᵀ b / ||Aᵀ(b - b')||. A normal-equation stop of the inner
    loop ends the call with that x (c = 0: M x = b is not solvable).
    """
    if tol_normal is None:
        tol_normal = tol
    b = np.asarray(b, dtype=np.float64)
    mtb = M.rmatvec(b)
    mtb_n2 = float(mtb @ mtb)
    x_best = np.array(x_eps, dtype=np.float64)
    rho_hi = float(np.linalg.norm(x_best))
    rho_lo = 0.0
    gap = tol * rho_hi
    wx = wbp = None
    used = trips = 0
    log = []
    status, reason = Status.OK, Reason.GAP
    while rho_hi - rho_lo > gap:
        if used >= max_iter:
            status, reason = Status.MAXITER, Reason.MAXITER
            break
        rho = 0.5 * (rho_hi + rho_lo)
        res = ta_fixed_rho(M, b, rho, wx, wbp, tol, tol_normal, max_iter - used,
                           recompute_every, mtb_n2)
        used += res.iters
        trips += 1
        if res.status == Status.OK and res.reason == Reason.RESIDUAL:
            rho_hi = rho
            x_best = res.x
        elif res.status == Status.WITNESS:
            rho_lo = res.db / res.cn
            wx, wbp = res.x, res.bp
        elif res.status == Status.OK and res.reason == Reason.NORMAL:
            x_best = res.x
            status, reason = Status.OK, Reason.NORMAL
            log.append((rho, int(res.status), int(res.reason), rho_hi, rho_lo, res.iters))
            break
        else:
            status, reason = res.status, res.reason
            log.append((rho, int(res.status), int(res.reason), rho_hi, rho_lo, res.iters))
            break
        log.append((rho, int(res.status), int(res.reason), rho_hi, rho_lo, res.iters))
    bn2 = float(b @ b)
    rt = b - M.matvec(x_best)
    nrt = M.rmatvec(rt)
    return MinNormResult(x_best, status, reason, rho_hi, rho_lo, trips, used, trip_log=log,
                         rel_res=math.sqrt(float(rt @ rt) / bn2),
                         rel_normal_res=math.sqrt(float(nrt @ nrt) / mtb_n2) if mtb_n2 > 0 else 0.0)


def ta_minnorm(A, b, tol=1e-10, tol_cta=None, tol_normal=None, max_iter=10000, t_max=5,
               cycle=PINGPONG, recompute_every=40) -> MinNormResult:
    """Hybrid CTA / TA of Sec. 5.2 for an approximate minimum-norm solution.

    1. CTA (Alg. 1.1) from x = 0 to tol_cta (default tol).
    2. If CTA's x satisfies ||b - A x|| <= tol_cta ||b|| the system is taken as
       solvable and Alg. 2.5 runs on (A, b); otherwise on (AᵀA, Aᵀb), applied
       through products with A and Aᵀ.
    max_iter bounds CTA iterations and TA iterations separately.
    """
    if tol_cta is None:
        tol_cta = tol
    if tol_normal is None:
        tol_normal = tol
    b = np.asarray(b, dtype=np.float64)
    if float(b @ b) == 0.0:
        return MinNormResult(np.zeros(A.n), Status.OK, Reason.ZERO_RHS, 0.0, 0.0, 0, 0,
                             rel_res=0.0, rel_normal_res=0.0)
    c = cta_solve(A, b, None, tol_cta, tol_normal, max_iter, t_max, cycle, recompute_every)
    if c.status not in (Status.OK,):
        return MinNormResult(c.x, c.status, c.reason, float(np.linalg.norm(c.x)), 0.0, 0, 0,
                             cta_iters=c.iters, rel_res=c.rel_res, rel_normal_res=c.rel_normal_res)
    if c.rel_res <= tol_cta:
        M, rhs, normal = A, b, False
    else:
        M, rhs, normal = NormalOperator(A), A.rmatvec(b), True
    r = ta_minnorm_bisect(M, rhs, c.x, tol, tol_normal, max_iter, recompute_every)
    r.cta_iters = c.iters
    r.normal_system = normal
    # report residuals of the original system A x = b
    bn2 = float(b @ b)
    atb = A.rmatvec(b)
    atbn2 = float(atb @ atb)
    rt = b - A.matvec(r.x)
    nrt = A.rmatvec(rt)
    r.rel_res = math.sqrt(float(rt @ rt) / bn2)
    r.rel_normal_res = math.sqrt(float(nrt @ nrt) / atbn2) if atbn2 > 0 else 0.0
    return r
