"""TA (Alg. 2.2 / 2.1, the LP form of Sec. 6, Alg. 2.5) on banded operands, whose products
take the run-staged kernels, against the oracle (needs a GB300)."""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle
from tests.test_gpu_fused_chain import CASES, dev, tacta  # noqa: F401  (shared cases and fixture)

pytestmark = pytest.mark.gpu



def banded_nonneg(m, n, offsets, seed):
    """A banded matrix with positive entries and b = A x+ for a seeded x+ >= 0 (an LP
    feasibility instance of Sec. 6 that is feasible by construction)."""
    rng = np.random.default_rng(seed)
    S = sp.diags([rng.uniform(0.5, 1.5, max(m, n)) for _ in offsets], offsets, shape=(m, n))
    S = sp.csr_matrix(S)
    S.sort_indices()
    b = S @ rng.uniform(0.0, 1.0, n)
    return gen.Problem(name="lp", m=m, n=n, fmt="csr", rowptr=S.indptr.astype(np.int32),
                       colidx=S.indices.astype(np.int32), vals=S.data.astype(np.float64), b=b)


def oracle_ta_spread(p, **opts):
    """How far the oracle's own TA trajectory moves when b is perturbed by 1e-16 relative
    noise (three seeded draws): the rounding sensitivity of the iteration on this system."""
    Ao = oracle.make_operator(p)
    ref = oracle.ta_solve(Ao, p.b, **opts)
    rng = np.random.default_rng(5)
    spread = 0.0
    for _ in range(3):
        r = oracle.ta_solve(Ao, p.b * (1 + 1e-16 * rng.standard_normal(p.m)), **opts)
        spread = max(spread, np.linalg.norm(r.x - ref.x) / np.linalg.norm(ref.x))
    return ref, spread


@pytest.mark.parametrize("name", list(CASES))
def test_ta_trajectory_matches_oracle(tacta, name):
    """100 TA iterations (Alg. 2.2) on banded operands: iterations, products, rho, x and
    the residual history against the oracle, to 1e-9 or ten times the oracle's own spread
    under 1e-16 perturbations of b, whichever is larger (TA on the 24 x 24 stencil moves by
    ~1e-7 under such perturbations, the other systems by < 1e-9)."""
    p = CASES[name]()
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=100)
    x, hist, info = tacta.ta_solve(A, b, **opts)
    ref, spread = oracle_ta_spread(p, **opts)
    tol = max(1e-9, 10 * spread)
    assert info["iters"] == ref.iters == 100 and info["matvecs"] == ref.matvecs
    assert info["rho"] == pytest.approx(ref.rho, rel=1e-9)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= tol * np.linalg.norm(ref.x), spread
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=max(1e-8, tol), atol=1e-13)


def test_ta_lp_feasibility_banded(tacta):
    """The LP form (c replaced by max(c, 0), Sec. 6) on a banded operand: a fixed trajectory
    against the oracle, then a feasible solve to 1e-6 with x >= 0 (A: 512 x 1500, diagonals
    at 0, 300, 700, three runs of x per tile)."""
    p = banded_nonneg(512, 1500, [0, 300, 700], 31)
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=25, nonneg=1)
    x, _, info = tacta.ta_solve(A, b, **opts)
    ref = oracle.ta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=25, nonneg=True)
    assert info["iters"] == ref.iters == 25
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    assert info["rho"] == pytest.approx(ref.rho, rel=1e-12)
    x, _, info = tacta.ta_solve(A, b, tol=1e-6, tol_normal=0.0, max_iter=400000, nonneg=1)
    xg = x.cpu().numpy()
    assert info["reason_name"] == "RESIDUAL" and info["rel_res"] <= 1e-6
    assert xg.min() >= 0.0
    S = sp.csr_matrix((p.vals, p.colidx, p.rowptr), shape=(p.m, p.n))
    assert np.linalg.norm(S @ xg - p.b) <= 1e-6 * np.linalg.norm(p.b) * (1 + 1e-9)


def test_ta_infeasible_lp_witness_banded(tacta):
    """b with negative entries against a nonnegative banded matrix: no x >= 0 solves
    A x = b, and the LP iteration stops with the Farkas certificate (reason WITNESS), as the
    oracle does."""
    p = banded_nonneg(2000, 2300, [0, 100], 32)
    p.b = p.b.copy()
    p.b[::7] = -1.0
    A, b = dev(p)
    opts = dict(tol=1e-8, tol_normal=1e-6, max_iter=100000, nonneg=1)
    _, _, info = tacta.ta_solve(A, b, **opts)
    ref = oracle.ta_solve(oracle.make_operator(p), p.b, tol=1e-8, tol_normal=1e-6, max_iter=100000, nonneg=True)
    assert ref.reason == oracle.Reason.WITNESS
    assert info["reason_name"] == "WITNESS"


def test_ta_minnorm_banded(tacta):
    """Algorithm 2.5 (trips of Alg. 2.1 at fixed rho) on a well-conditioned banded
    underdetermined system: the gap closes (reason GAP) and x is the minimum-norm solution
    within 50 tol, as the oracle's is."""
    rng = np.random.default_rng(41)
    S = sp.csr_matrix(sp.diags([3.0 + rng.uniform(0, 1, 1200), rng.uniform(-0.5, 0.5, 1200),
                                rng.uniform(-0.5, 0.5, 1200)], [0, 60, 150], shape=(1200, 1400)))
    S.sort_indices()
    b = S @ rng.standard_normal(1400)
    p = gen.Problem(name="mn", m=1200, n=1400, fmt="csr", rowptr=S.indptr.astype(np.int32),
                    colidx=S.indices.astype(np.int32), vals=S.data.astype(np.float64), b=b)
    A, bd = dev(p)
    tol = 1e-6
    kw = dict(tol=tol, tol_cta=1e-10, tol_normal=0.0, max_iter=2000000)
    x, _, info = tacta.ta_minnorm(A, bd, **kw)
    ref = oracle.ta_minnorm(oracle.make_operator(p), p.b, **kw)
    xs = np.linalg.lstsq(S.toarray(), b, rcond=None)[0]
    assert info["reason_name"] == "GAP" and ref.reason == oracle.Reason.GAP
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 50 * tol * np.linalg.norm(xs)
    assert np.linalg.norm(ref.x - xs) <= 50 * tol * np.linalg.norm(xs)
