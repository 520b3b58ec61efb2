"""Rounding spread of the oracle itself (test helper, imported by the GPU parity tests).

Two correct FP64 implementations that add in different orders follow CTA / TA
trajectories that agree for tens of steps and then drift apart, so the step at which a
run to tolerance stops is itself rounding-sensitive. The oracle shows how much: it is
run on right-hand sides perturbed by 1e-16 relative noise (seeded), in a pool of spawned
worker processes (numpy and the oracle only: no CUDA in the workers).

stop_index_window gives the window a GPU stop index must fall in: Tukey's outlier fences
of the oracle's stop indices over those runs and the unperturbed one (1.5 interquartile
ranges beyond the quartiles, which hold 99.3% of a normal distribution), widened to the
sample range and by one step either way. When the oracle's index does not move, the
window is the unperturbed index +- 1.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

SAMPLES = 16
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _perturbed(b, seed):
    return b * (1.0 + 1e-16 * np.random.default_rng(seed).standard_normal(b.size))


def _stop_index(args):
    solve_name, p, x0, okw, seed = args
    import oracle
    solve = getattr(oracle, solve_name)
    b = p.b if seed is None else _perturbed(p.b, seed)
    return int(solve(oracle.make_operator(p), b, x0, **okw).iters)


def _bisect_log(args):
    p, rhs, normal, x_eps, okw, seed = args
    import oracle
    from oracle.ta import ta_minnorm_bisect
    A = oracle.make_operator(p)
    M = oracle.NormalOperator(A) if normal else A
    b = rhs if seed is None else _perturbed(rhs, seed)
    r = ta_minnorm_bisect(M, b, x_eps, **okw)
    return [(int(row[2]), int(row[5])) for row in r.trip_log]


def _map(fn, jobs):
    """fn over jobs in spawned workers with one BLAS thread each."""
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    try:
        for k in _THREAD_VARS:
            os.environ[k] = "1"
        workers = max(1, min(len(jobs), os.cpu_count() or 1))
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(fn, jobs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def stop_index_window(solve_name, p, x0, okw, n=SAMPLES):
    """(lo, hi, indices): the window for a stop index of oracle.<solve_name> on problem p
    from x0 with options okw; indices[0] is the unperturbed run."""
    jobs = [(solve_name, p, x0, okw, None)] + [(solve_name, p, x0, okw, 1000 + i) for i in range(n)]
    its = np.array(_map(_stop_index, jobs))
    q1, q3 = np.percentile(its, [25, 75])
    iqr = q3 - q1
    lo = min(its.min(), int(np.floor(q1 - 1.5 * iqr))) - 1
    hi = max(its.max(), int(np.ceil(q3 + 1.5 * iqr))) + 1
    return lo, hi, its


def _bisect_x(args):
    p, rhs, normal, x_eps, okw, seed = args
    import oracle
    from oracle.ta import ta_minnorm_bisect
    A = oracle.make_operator(p)
    M = oracle.NormalOperator(A) if normal else A
    b = rhs if seed is None else _perturbed(rhs, seed)
    return ta_minnorm_bisect(M, b, x_eps, **okw).x


def bisect_x_spread(p, rhs, normal, x_eps, okw, n=4):
    """Largest relative distance between the oracle's Algorithm 2.5 answer on rhs and on n
    perturbed right-hand sides (the rounding growth of its TA trips)."""
    jobs = [(p, rhs, normal, x_eps, okw, None)] + [(p, rhs, normal, x_eps, okw, 3000 + i) for i in range(n)]
    xs = _map(_bisect_x, jobs)
    nx = np.linalg.norm(xs[0])
    return max(np.linalg.norm(x - xs[0]) for x in xs[1:]) / (nx if nx > 0 else 1.0)


def stable_trip_prefix(p, rhs, normal, x_eps, okw, n=8):
    """Number of leading trips of Algorithm 2.5 whose (stop reason, iterations) the oracle
    reproduces on every one of n perturbed right-hand sides, and the unperturbed log."""
    jobs = [(p, rhs, normal, x_eps, okw, None)] + [(p, rhs, normal, x_eps, okw, 2000 + i) for i in range(n)]
    logs = _map(_bisect_log, jobs)
    k = 0
    while all(len(lg) > k and lg[k] == logs[0][k] for lg in logs):
        k += 1
    return k, logs[0]
