"""Algorithm 2.5 (Sec. 4.4) trip by trip against the oracle, through the C ABI.

tacta_plan_minnorm_bisect and oracle.ta.ta_minnorm_bisect run the bisection on rho from
the same approximate solution x_eps. A trip of Alg. 2.1 that runs to the residual test
takes a rounding-sensitive number of TA iterations once it is long, so the comparison is
made on the trips the oracle itself reproduces under 1e-16 perturbations of b
(tests/oracle_spread.stable_trip_prefix): when every trip is reproducible the whole
bisection is compared; otherwise max_iter is set to the iterations of the reproducible
trips plus one, so that both sides stop (MAXITER) one iteration into the first trip that
is not. Per trip: the same stop reason and iteration count, rho, rho_hi and rho_lo to
1e-10; the final x to 1e-9 (the task's FP64 tolerance) or, where the oracle's own answer
moves more than that under the perturbations (TA trips of ~30 iterations from a witness
amplify rounding to ~1e-9), ten times the oracle's own spread.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle.ta import ta_minnorm_bisect
from tests.oracle_spread import bisect_x_spread, stable_trip_prefix

pytestmark = pytest.mark.gpu

X_TOL = 1e-9
RHO_TOL = 1e-10


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def _plan(tacta, p):
    import torch
    d = torch.device("cuda:0")
    A = tacta.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n))
    return tacta.Plan(A)


def _compare(tacta, p, x_eps, normal, tol, min_trips):
    import torch
    Ao = oracle.make_operator(p)
    rhs = Ao.rmatvec(p.b) if normal else p.b
    okw = dict(tol=tol, tol_normal=0.0, max_iter=200000)
    k, log0 = stable_trip_prefix(p, rhs, normal, x_eps, okw)
    assert k >= min_trips, (k, log0)          # the case exercises several trips
    if k < len(log0):
        okw["max_iter"] = sum(it for _, it in log0[:k]) + 1
    M = oracle.NormalOperator(Ao) if normal else Ao
    ref = ta_minnorm_bisect(M, rhs, x_eps, **okw)
    plan = _plan(tacta, p)
    try:
        d = torch.device("cuda:0")
        x, log, info = plan.minnorm_bisect(torch.from_numpy(p.b).to(d), torch.from_numpy(x_eps).to(d),
                                           normal=normal, **okw)
    finally:
        plan.close()
    ref_log = np.array([row for row in ref.trip_log], dtype=np.float64)
    assert info["trips"] == ref.trips == len(ref_log), (info["trips"], ref.trips)
    assert info["reason"] == int(ref.reason)
    for i, (g, r) in enumerate(zip(log, ref_log)):
        # oracle row: (rho, status, reason, rho_hi, rho_lo, iters); device row:
        # (rho, reason, rho_hi, rho_lo, iters, 0)
        assert int(g[1]) == int(r[2]) and int(g[4]) == int(r[5]), (i, g, r)
        assert g[0] == pytest.approx(r[0], rel=RHO_TOL), i
        assert g[2] == pytest.approx(r[3], rel=RHO_TOL), i
        assert g[3] == pytest.approx(r[4], rel=RHO_TOL, abs=RHO_TOL * r[3]), i
    assert info["rho"] == pytest.approx(ref.rho_upper, rel=RHO_TOL)
    assert info["rho_lower"] == pytest.approx(ref.rho_lower, rel=RHO_TOL, abs=RHO_TOL * ref.rho_upper)
    xg = x.cpu().numpy()
    err = np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)
    if err > X_TOL:
        spread = bisect_x_spread(p, rhs, normal, x_eps, okw)
        assert err <= 10 * spread, (err, spread)
    assert info["iters"] == ref.iters
    return log, ref, k


@pytest.mark.parametrize("m,n", [(300, 500), (12000, 20000)])
def test_bisection_trip_by_trip_whole_run(tacta, m, n):
    """Banded full-row-rank systems, x_eps = the generating x (not minimum-norm): the six
    trips of the tol = 1e-2 bisection alternate witnesses and successes; the larger one
    (12,000 rows, 47 row tiles per product) runs on the tiled device products."""
    p = gen.banded_rect(m, n)
    log, ref, k = _compare(tacta, p, p.x_known, False, 1e-2, min_trips=5)
    assert int(ref.reason) == 6                 # GAP: the whole bisection was compared
    reasons = {int(r[1]) for r in log}
    assert reasons == {1, 5}                    # both outcomes of Alg. 2.1 occur


def test_bisection_trip_by_trip_truncated(tacta):
    """At tol = 3e-3 the later success trips run long enough to become rounding-sensitive:
    the reproducible prefix is compared and both sides stop one iteration into the next."""
    p = gen.banded_rect(12000, 20000)
    log, ref, k = _compare(tacta, p, p.x_known, False, 3e-3, min_trips=4)
    assert int(ref.reason) in (3, 6)            # MAXITER after the prefix, or the whole run


def test_bisection_on_the_normal_equation(tacta):
    """Tall inconsistent system: Alg. 2.5 on (AᵀA, Aᵀb) applied through products with A
    and Aᵀ, from x_eps = the generating x plus noise."""
    q = gen.banded_rect(300, 500)
    # the transpose: 500 x 300, b not in its range
    S = q.scipy().T.tocsr()
    S.sort_indices()
    rng = np.random.default_rng(9)
    b = rng.standard_normal(500)
    p = gen.Problem("banded_T", 500, 300, "csr", None, S.indptr.astype(np.int32),
                    S.indices.astype(np.int32), S.data.astype(np.float64), b=b)
    x_ls = np.linalg.lstsq(p.to_dense(), b, rcond=None)[0]
    x_eps = x_ls + 0.3 * rng.standard_normal(300)
    _compare(tacta, p, x_eps, True, 1e-2, min_trips=2)


def test_bisection_zero_rhs_and_arguments(tacta):
    import torch
    p = gen.banded_rect(30, 50)
    plan = _plan(tacta, p)
    try:
        d = torch.device("cuda:0")
        z = torch.zeros(30, dtype=torch.float64, device=d)
        x, log, info = plan.minnorm_bisect(z, torch.ones(50, dtype=torch.float64, device=d), tol=1e-3)
        assert info["reason_name"] == "ZERO_RHS" and not x.any() and len(log) == 0
        with pytest.raises(ValueError):
            plan.minnorm_bisect(torch.from_numpy(p.b).to(d), np.ones(50), tol=1e-3)
    finally:
        plan.close()
