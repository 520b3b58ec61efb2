"""The rounding-spread helper the GPU parity tests use (CPU: the oracle only)."""
import numpy as np

import gen
import oracle
from tests.oracle_spread import stable_trip_prefix, stop_index_window


def test_stop_index_window_holds_the_unperturbed_index_and_every_sample():
    p = gen.convdiff_stencil(7)
    okw = dict(tol=1e-12, tol_normal=0.0, max_iter=20000)
    lo, hi, its = stop_index_window("cta_solve", p, None, okw)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, None, **okw).iters
    assert its[0] == ref and len(its) == 17
    assert lo < its.min() <= its.max() < hi
    # a run whose stop index does not move under the perturbations: the window is +-1
    q = gen.dense_gaussian(40, 300, seed=5)
    lo, hi, its = stop_index_window("cta_solve", q, None, dict(tol=1e-11, tol_normal=0.0, max_iter=5000))
    assert np.all(its == its[0]) and (lo, hi) == (its[0] - 1, its[0] + 1)


def test_stable_trip_prefix_of_a_short_bisection():
    p = gen.banded_rect(300, 500)
    k, log0 = stable_trip_prefix(p, p.b, False, p.x_known, dict(tol=1e-2, tol_normal=0.0, max_iter=200000))
    assert k == len(log0) >= 5
    assert {r for r, _ in log0} == {1, 5}
