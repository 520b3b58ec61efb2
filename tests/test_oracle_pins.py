"""Pins of the FP64 oracle to the paper and to textbook mathematics (CPU only).

Nothing here compares the oracle with itself or with the CUDA path: every
expected value is a closed form or theorem from the paper, a hand-derived
fixture under tests/golden/, a brute-force definition, or an independent
library routine (SVD least squares, pinv, LSQR).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import gen
import oracle
from oracle import Status, Reason

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def op_dense(A):
    A = np.asarray(A, dtype=np.float64)
    return oracle.Operator(A.shape[0], A.shape[1], "dense", dense=A)


def op_csr(p):
    return oracle.make_operator(p)


def minnorm(A, b, rcond=1e-10):
    """A⁺ b by a rank-truncated SVD (independent of the oracle)."""
    return np.linalg.pinv(np.asarray(A), rcond=rcond) @ b


# --------------------------------------------------------------------------- products

def test_csr_products_are_the_definition():
    """(A x)_i and (Aᵀ r)_j against a brute-force double loop; ragged and empty rows."""
    p = gen.random_csr(23, 17, density=0.2, seed=5, empty_rows=4, long_rows=2)
    A = op_csr(p)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(p.n)
    r = rng.standard_normal(p.m)
    y = np.zeros(p.m)
    z = np.zeros(p.n)
    for i in range(p.m):
        for k in range(p.rowptr[i], p.rowptr[i + 1]):
            y[i] += p.vals[k] * x[p.colidx[k]]
            z[p.colidx[k]] += p.vals[k] * r[i]
    np.testing.assert_allclose(A.matvec(x), y, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(A.rmatvec(r), z, rtol=1e-14, atol=1e-14)
    D = p.to_dense()
    np.testing.assert_allclose(op_dense(D).matvec(x), y, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(op_dense(D).rmatvec(r), z, rtol=1e-13, atol=1e-13)


def test_normal_operator_is_AtA():
    rng = np.random.default_rng(1)
    D = rng.standard_normal((7, 11))
    M = oracle.NormalOperator(op_dense(D))
    x = rng.standard_normal(11)
    np.testing.assert_allclose(M.matvec(x), D.T @ (D @ x), rtol=1e-13)
    assert M.m == M.n == 11


# --------------------------------------------------------------------------- schedule

def test_schedule_matches_sec51_cycling():
    g = golden("schedule_pingpong.json")
    got = [oracle.schedule(k, g["t_max"], oracle.PINGPONG) for k in range(len(g["orders"]))]
    assert got == g["orders"]
    assert [oracle.schedule(k, 3, oracle.SAWTOOTH) for k in range(7)] == [1, 2, 3, 1, 2, 3, 1]
    assert [oracle.schedule(k, 4, oracle.FIXED) for k in range(3)] == [4, 4, 4]
    assert [oracle.schedule(k, 1, oracle.PINGPONG) for k in range(3)] == [1, 1, 1]
    assert [oracle.schedule(k, 2, oracle.PINGPONG) for k in range(5)] == [1, 2, 1, 2, 1]


# --------------------------------------------------------------------------- auxiliary equation

def test_hankel_golden_closed_forms():
    """Ex. exam1: alpha_{1,1} = phi1/phi2 and the two t = 2 formulas (golden values)."""
    g = golden("hankel_t2.json")
    a1, r1 = oracle.hankel_solve(g["phi"], 1)
    a2, r2 = oracle.hankel_solve(g["phi"], 2)
    assert r1 == 1 and r2 == 2
    np.testing.assert_allclose(a1, g["alpha_t1"], rtol=1e-14)
    np.testing.assert_allclose(a2, g["alpha_t2"], rtol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_hankel_closed_forms_random(seed):
    """Ex. exam1 closed forms on moments phi_i = rᵀ H^i r of random SPD H."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((6, 6))
    H = B @ B.T + 0.5 * np.eye(6)
    r = rng.standard_normal(6)
    phi = [0.0] + [float(r @ np.linalg.matrix_power(H, i) @ r) for i in range(1, 5)]
    a, _ = oracle.hankel_solve(phi, 1)
    assert a[0] == pytest.approx(phi[1] / phi[2], rel=1e-14)
    den = phi[2] * phi[4] - phi[3] ** 2
    a, rank = oracle.hankel_solve(phi, 2)
    assert rank == 2
    assert a[0] == pytest.approx((phi[1] * phi[4] - phi[2] * phi[3]) / den, rel=1e-9)
    assert a[1] == pytest.approx((phi[2] ** 2 - phi[1] * phi[3]) / den, rel=1e-9)


def test_hankel_zero_moments_breakdown():
    """H r = 0 gives phi_2 = 0: no step (Ex. exam1: then x solves the normal equation)."""
    alpha, rank = oracle.hankel_solve([0.0, 0.0, 0.0, 0.0, 0.0], 2)
    assert rank == 0 and alpha == [0.0, 0.0]


@pytest.mark.parametrize("t", [1, 2, 3, 4, 5])
def test_Ft_is_the_least_squares_step(t):
    """Eq. F_t: alpha minimises ||r - sum alpha_i H^i r||. Compare r'' with an SVD
    least-squares solve over the Krylov block [H r, ..., H^t r]."""
    rng = np.random.default_rng(10 + t)
    # singular values in [0.6, 1.4]: the power basis of H stays well conditioned up to t = 5
    Q1, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    Q2, _ = np.linalg.qr(rng.standard_normal((9, 9)))
    D = Q1[:, :9] @ np.diag(np.linspace(0.6, 1.4, 9)) @ Q2.T
    A = op_dense(D)
    H = D @ D.T
    r = rng.standard_normal(12)
    K = np.stack([np.linalg.matrix_power(H, i) @ r for i in range(1, t + 1)], axis=1)
    coef, *_ = np.linalg.lstsq(K, r, rcond=None)
    r_ls = r - K @ coef
    x2, r2, alpha, rank, phi = oracle.cta_step(A, np.zeros(9), r, t)
    assert rank == t
    # optimality: r_ls is the minimiser, so ||r''|| can only match it
    assert np.linalg.norm(r2) <= np.linalg.norm(r_ls) * (1 + 1e-12)
    np.testing.assert_allclose(r2, r_ls, rtol=0, atol=1e-9 * np.linalg.norm(r))
    # x'' = x' + sum alpha_i Aᵀ H^{i-1} r'  (Eq. CTAGEN7A, H = A Aᵀ)
    xs = sum(alpha[i] * (D.T @ np.linalg.matrix_power(H, i) @ r) for i in range(t))
    np.testing.assert_allclose(x2, xs, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("t", [1, 2, 3, 5])
def test_Ft_equals_t_lsqr_steps(t):
    """Textbook equivalence: F_t with H = A Aᵀ from x' minimises ||b - A x|| over
    x' + span{Aᵀr', (AᵀA)Aᵀr', ...}, as do t iterations of LSQR from x'."""
    rng = np.random.default_rng(20 + t)
    Q1, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    Q2, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    D = Q1[:, :20] @ np.diag(np.linspace(0.5, 2.0, 20)) @ Q2.T
    b = rng.standard_normal(30)
    x0 = rng.standard_normal(20)
    A = op_dense(D)
    x2, r2, *_ = oracle.cta_step(A, x0, b - D @ x0, t)
    ls = spla.lsqr(D, b, x0=x0, iter_lim=t, atol=0, btol=0, conlim=0)[0]
    np.testing.assert_allclose(x2, ls, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(r2, b - D @ x2, rtol=1e-10, atol=1e-10)


def test_F1_residual_ratio_identity():
    """Thm. thmdynamic (ii), Eq. subseceq3.4: ||r_{k+1}||²/||r_k||² = 1 - phi1²/(phi2 ||r_k||²)."""
    rng = np.random.default_rng(3)
    D = rng.standard_normal((15, 15))
    A = op_dense(D)
    r = rng.standard_normal(15)
    x = np.zeros(15)
    for _ in range(8):
        x2, r2, alpha, rank, phi = oracle.cta_step(A, x, r, 1)
        lhs = (r2 @ r2) / (r @ r)
        rhs = 1.0 - phi[1] ** 2 / (phi[2] * (r @ r))
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-14)
        assert lhs < 1.0
        x, r = x2, r2


def test_F1_eigenvector_start_converges_in_one_step():
    """Thm. thmdynamic (iii): r_0 an eigenvector of H => r_1 = F_1(r_0) = 0."""
    a = np.array([0.5, 1.0, 2.0, 3.0])
    A = op_dense(np.diag(a))
    for j in range(4):
        b = np.zeros(4)
        b[j] = 1.7
        x2, r2, *_ = oracle.cta_step(A, np.zeros(4), b, 1)
        assert np.linalg.norm(r2) <= 1e-15
        assert x2[j] == pytest.approx(1.7 / a[j], rel=1e-15)


def test_critical_line_zigzag_golden():
    """Thm. thmdynamic (iv): on the ij-critical line F_1 maps r+ to rho r- and back."""
    g = golden("critical_lines_2x2.json")
    A = op_dense(np.diag(g["A_diag"]))
    r = np.array(g["r_plus"])
    x = np.zeros(2)
    for k, want in enumerate(g["orbit_first_steps"]):
        np.testing.assert_allclose(r, want, rtol=1e-13, atol=1e-15)
        assert np.linalg.norm(r) == pytest.approx(g["rho"] ** k, rel=1e-13)
        x, r, *_ = oracle.cta_step(A, x, r, 1)
    # the convex combination alpha_* r_0 + (1 - alpha_*) r_1 is an eigenvector: F_1 kills it
    r0 = np.array(g["r_plus"])
    _, r1, *_ = oracle.cta_step(A, np.zeros(2), r0, 1)
    bar = g["alpha_star"] * r0 + (1 - g["alpha_star"]) * r1
    np.testing.assert_allclose(bar, g["convex_point"], rtol=1e-13, atol=1e-15)
    _, rb, *_ = oracle.cta_step(A, np.zeros(2), bar, 1)
    assert np.linalg.norm(rb) <= 1e-15


@pytest.mark.parametrize("i,j", [(0, 3), (1, 2), (0, 4)])
def test_critical_line_rate_mxm(i, j):
    """Eq. c-three: ||r_k|| = rho_ij^k ||r_0|| on the ij-critical line of an m x m diagonal H."""
    a = np.array([1.0, 1.5, 2.0, 2.5, 4.0])
    lam = a ** 2
    A = op_dense(np.diag(a))
    ai = math.sqrt(lam[j] / (lam[i] + lam[j]))
    aj = math.sqrt(lam[i] / (lam[i] + lam[j]))
    rho = (lam[j] - lam[i]) / (lam[j] + lam[i])
    r = np.zeros(5)
    r[i], r[j] = ai, aj
    x = np.zeros(5)
    for k in range(1, 12):
        x, r, *_ = oracle.cta_step(A, x, r, 1)
        assert np.linalg.norm(r) == pytest.approx(rho ** k, rel=1e-10)


def _svd_matrix(rng, m, n, svals):
    """m x n matrix with the given singular values and random singular vectors."""
    k = len(svals)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q1[:, :k] @ np.diag(svals) @ Q2[:, :k].T


@pytest.mark.parametrize("seed", range(4))
def test_pointwise_orbit_theorem(seed):
    """Thm. on point-wise orbits (i)-(iii): ||F_1(r0)|| > ... > ||F_s(r0)||; the
    system is solvable iff F_s(r0) = 0; otherwise Aᵀ F_s(r0) = 0.
    (Singular values are kept in [0.7, 1.6] so the t = 5 power basis of H is
    resolvable in FP64; with a spread of 1e4 the fifth moment direction falls
    below double precision and the truncated solve drops it.)"""
    rng = np.random.default_rng(40 + seed)
    m = 5
    D = _svd_matrix(rng, m, m, np.linspace(0.7, 1.6, m))
    A = op_dense(D)
    b = rng.standard_normal(m)
    norms = [np.linalg.norm(oracle.cta_step(A, np.zeros(m), b, t)[1]) for t in range(1, m + 1)]
    assert all(norms[t] < norms[t - 1] for t in range(1, m))
    assert norms[-1] <= 1e-8 * np.linalg.norm(b)            # solvable: F_s(r0) = 0
    # rank-deficient, b outside the range: F_s(r0) != 0 but Aᵀ F_s(r0) = 0
    Dr = _svd_matrix(rng, m, m, [0.8, 1.2, 1.5])
    br = rng.standard_normal(m)
    Ar = op_dense(Dr)
    x2, r2, *_ = oracle.cta_step(Ar, np.zeros(m), br, 3)      # s = rank = 3 for H = Dr Drᵀ
    assert np.linalg.norm(r2) > 1e-3 * np.linalg.norm(br)
    assert np.linalg.norm(Dr.T @ r2) <= 1e-8 * np.linalg.norm(Dr.T @ br)


def test_truncated_solve_drops_unresolvable_direction():
    """Reading of the min-norm auxiliary solve: when H^t r adds no direction that FP64
    can resolve, the leading block is solved and the residual still decreases."""
    rng = np.random.default_rng(43)
    D = _svd_matrix(rng, 5, 5, [3.9, 1.8, 1.5, 0.98, 0.028])
    A = op_dense(D)
    b = rng.standard_normal(5)
    norms, ranks = [], []
    for t in range(1, 6):
        _, r2, _, rank, _ = oracle.cta_step(A, np.zeros(5), b, t)
        norms.append(np.linalg.norm(r2))
        ranks.append(rank)
    assert ranks[:4] == [1, 2, 3, 4]
    assert all(norms[t] <= norms[t - 1] * (1 + 1e-12) for t in range(1, 5))


# --------------------------------------------------------------------------- CTA solves

def test_cta_min_norm_limit_low_rank_square():
    """Thm. thmone (4): from x0 = 0, x_k ∈ range(Aᵀ), and the limit is A⁺ b."""
    p = gen.dense_low_rank(64, 64, 32, seed=1)
    A = op_dense(p.dense)
    res = oracle.cta_solve(A, p.b, tol=1e-12, tol_normal=0.0, max_iter=20000)
    assert res.status == Status.OK and res.reason == Reason.RESIDUAL
    xs = minnorm(p.dense, p.b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-9
    P = np.linalg.pinv(p.dense, rcond=1e-10) @ p.dense        # projector onto range(Aᵀ)
    assert np.linalg.norm(res.x - P @ res.x) <= 1e-9 * np.linalg.norm(res.x)
    assert res.rel_res <= 1e-12


def test_cta_min_norm_underdetermined():
    rng = np.random.default_rng(7)
    D = rng.standard_normal((40, 90))
    b = D @ rng.standard_normal(90)
    res = oracle.cta_solve(op_dense(D), b, tol=1e-12, tol_normal=0.0, max_iter=20000)
    assert res.reason == Reason.RESIDUAL
    xs = minnorm(D, b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-10


def test_cta_range_invariant_every_step():
    """Thm. thmone (4): every iterate lies in range(Aᵀ) (checked after each step)."""
    p = gen.dense_low_rank(24, 30, 10, seed=2)
    P = np.linalg.pinv(p.dense, rcond=1e-10) @ p.dense
    bad = []

    def obs(k, x, r, t, alpha, rank, phi):
        if np.linalg.norm(x - P @ x) > 1e-10 * max(1.0, np.linalg.norm(x)):
            bad.append(k)
    oracle.cta_solve(op_dense(p.dense), p.b, tol=1e-11, tol_normal=0.0, max_iter=300, observer=obs)
    assert not bad


def test_cta_stencil_recovers_ones():
    """Sec. 5.1 convention b = A·1: the nonsingular stencil system has x* = 1."""
    p = gen.convdiff_stencil(12)
    res = oracle.cta_solve(op_csr(p), p.b, tol=1e-12, tol_normal=0.0, max_iter=20000)
    assert res.reason == Reason.RESIDUAL
    assert np.abs(res.x - 1.0).max() < 1e-9
    assert res.rel_res <= 1e-12


def test_stencil_matches_its_definition():
    """Row (i, j) of the stencil: 4 centre, -1 -+ beta h/2 neighbours (cell Péclet 0.5)."""
    N = 5
    p = gen.convdiff_stencil(N)
    D = p.to_dense()
    for j in range(N):
        for i in range(N):
            row = j * N + i
            want = np.zeros(N * N)
            want[row] = 4.0
            if i > 0:
                want[row - 1] = -1.5
            if i < N - 1:
                want[row + 1] = -0.5
            if j > 0:
                want[row - N] = -1.25
            if j < N - 1:
                want[row + N] = -0.75
            np.testing.assert_array_equal(D[row], want)
    assert p.nnz == 5 * N * N - 4 * N


def clement_minnorm_closed_form(n):
    """A⁺ 1-row-sum solution of the odd Clement matrix: b = A·1 so A⁺b = 1 - (1ᵀv/||v||²) v,
    v the null vector (even entries 0, odd entries v_{i+1} = -(c_{i-1}/c_i) v_{i-1})."""
    c = np.sqrt(np.arange(1, n) * (n - np.arange(1, n)))      # c[i-1] = c_i, 1-based i
    v = np.zeros(n)
    v[0] = 1.0
    for i in range(2, n, 2):       # 1-based row i (even) gives v_{i+1} from v_{i-1}
        v[i] = -(c[i - 2] / c[i - 1]) * v[i - 2]
    one = np.ones(n)
    return one - (one @ v) / (v @ v) * v, v


def test_clement_spectrum_and_null_vector():
    g = golden("clement_spectrum.json")
    for n, key in ((5, "n5"), (6, "n6")):
        ev = np.sort(np.linalg.eigvalsh(gen.clement(n).to_dense()))
        np.testing.assert_allclose(ev, g[key], atol=1e-12)
    n = 41
    D = gen.clement(n).to_dense()
    xs, v = clement_minnorm_closed_form(n)
    assert np.linalg.norm(D @ v) <= 1e-12 * np.linalg.norm(v)
    np.testing.assert_allclose(xs, minnorm(D, D @ np.ones(n)), rtol=1e-9, atol=1e-9)


def test_cta_clement_min_norm():
    """Singular Clement, b = A·1 in range(A): CTA from 0 reaches A⁺b (Thm. thmone (4))."""
    n = 201
    p = gen.clement(n)
    res = oracle.cta_solve(op_csr(p), p.b, tol=1e-12, tol_normal=0.0, max_iter=50000)
    assert res.reason == Reason.RESIDUAL
    xs, _ = clement_minnorm_closed_form(n)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-9


def test_cta_inconsistent_stops_on_normal_equation():
    """b ∉ range(A): ||r|| cannot reach tol; the normal-equation clause stops CTA
    (Alg. 1.1) and x approximates the minimum-norm least-squares solution."""
    p = gen.dense_low_rank(30, 30, 12, seed=4)
    rng = np.random.default_rng(4)
    b = p.b + rng.standard_normal(30)
    res = oracle.cta_solve(op_dense(p.dense), b, tol=1e-12, tol_normal=1e-12, max_iter=20000)
    assert res.status == Status.OK and res.reason == Reason.NORMAL
    xs = minnorm(p.dense, b)
    assert np.linalg.norm(res.x - xs) / np.linalg.norm(xs) < 1e-8
    assert res.rel_res > 1e-3


def test_cta_recompute_makes_history_the_true_residual():
    """At every multiple of R the carried residual is b - A x (reading of Eq. CTAGEN7)."""
    p = gen.convdiff_stencil(8)
    A = op_csr(p)
    seen = {}

    def obs(k, x, r, t, alpha, rank, phi):
        if k % 5 == 0:
            seen[k] = np.linalg.norm(r - (p.b - p.scipy() @ x))
    oracle.cta_solve(A, p.b, tol=1e-30, tol_normal=0.0, max_iter=20, recompute_every=5, observer=obs)
    assert seen and max(seen.values()) == 0.0


def test_cta_zero_rhs_and_maxiter():
    p = gen.convdiff_stencil(6)
    res = oracle.cta_solve(op_csr(p), np.zeros(p.m), tol=1e-10)
    assert res.reason == Reason.ZERO_RHS and not res.x.any()
    res = oracle.cta_solve(op_csr(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=7)
    assert res.status == Status.MAXITER and res.iters == 7 and len(res.hist) == 8
    # per-step orders follow the schedule: 1+2+3+4+5+4+3 products pairs + Aᵀb
    assert res.matvecs == 1 + 2 * sum(oracle.schedule(k, 5) for k in range(7))


def test_cta_residual_monotone():
    """Each F_t reduces the residual (Ex. exam1: ||F(r0)|| < ||r0|| when H r0 != 0)."""
    p = gen.clement(51)
    res = oracle.cta_solve(op_csr(p), p.b, tol=1e-13, tol_normal=0.0, max_iter=200, recompute_every=0)
    h = np.array(res.hist)
    assert np.all(np.diff(h) <= 1e-15)


# --------------------------------------------------------------------------- TA

def test_ta_identity_golden():
    g = golden("ta_identity.json")
    A = op_dense(g["A"])
    rhos = []
    res = oracle.ta_solve(A, np.array(g["b"]), tol=1e-14, max_iter=10,
                          observer=lambda k, x, bp, rho, a: rhos.append(rho))
    assert rhos[0] == g["rho_after_1"]
    assert res.iters == g["iters"] and res.reason == Reason.RESIDUAL
    np.testing.assert_allclose(res.x, g["x_after_2"], rtol=1e-15)


def test_ta_invariants_each_iteration():
    """Alg. 2.2: ||x'|| <= rho, b' = A x' (carried), alpha in (0, 1] (Prop. prop1TA)."""
    p = gen.dense_gaussian(20, 30, seed=3)
    D = p.dense
    bad = []

    def obs(k, x, bp, rho, alpha):
        if np.linalg.norm(x) > rho * (1 + 1e-12):
            bad.append(("norm", k))
        if np.linalg.norm(bp - D @ x) > 1e-10 * np.linalg.norm(bp):
            bad.append(("drift", k))
        if alpha is not None and not (0.0 < alpha <= 1.0):
            bad.append(("alpha", k))
    res = oracle.ta_solve(op_dense(D), p.b, tol=1e-6, max_iter=5000, observer=obs)
    assert not bad
    assert res.status == Status.OK


def test_ta_converges_consistent():
    """Thm. finalthm (i): Alg. 2.2 reaches an eps-approximate solution with ||x|| <= rho."""
    rng = np.random.default_rng(8)
    D = rng.standard_normal((10, 25))
    b = D @ rng.standard_normal(25)
    res = oracle.ta_solve(op_dense(D), b, tol=1e-8, tol_normal=0.0, max_iter=200000)
    assert res.reason == Reason.RESIDUAL
    assert res.rel_res <= 1e-8 * (1 + 1e-9)
    assert np.linalg.norm(res.x) <= res.rho * (1 + 1e-12)


def test_ta_witness_lower_bound():
    """Alg. 2.1 at rho < ||x_*|| stops on a witness with (b-b')ᵀb/||c|| < ||x_*|| (Cor. cor1);
    at rho = 2 ||x_*|| it finds an approximate solution."""
    rng = np.random.default_rng(9)
    D = rng.standard_normal((8, 12))
    b = D @ rng.standard_normal(12)
    xs = minnorm(D, b)
    nx = np.linalg.norm(xs)
    A = op_dense(D)
    w = oracle.ta_fixed_rho(A, b, 0.5 * nx, tol=1e-8, max_iter=100000)
    assert w.status == Status.WITNESS
    assert w.db / w.cn < nx
    assert w.db / w.cn > 0.5 * nx                      # the bound improves on rho itself
    ok = oracle.ta_fixed_rho(A, b, 2.0 * nx, tol=1e-6, tol_normal=0.0, max_iter=200000)
    assert ok.status == Status.OK and ok.reason == Reason.RESIDUAL
    assert np.linalg.norm(ok.x) <= 2.0 * nx * (1 + 1e-12)


def test_ta_minnorm_bisection_consistent():
    """Alg. 2.5: rho_lo <= ||x_*|| (Cor. cor1), exits with the gap closed, and the answer
    is an eps-approximate minimum-norm solution (Def. minnormapp, Prop. propx)."""
    rng = np.random.default_rng(11)
    D = rng.standard_normal((6, 10))
    b = D @ rng.standard_normal(10)
    xs = minnorm(D, b)
    nx = np.linalg.norm(xs)
    x_eps = xs + 0.3 * rng.standard_normal(10) * np.linalg.norm(xs) / 10   # a worse start
    x_eps = x_eps - minnorm(D, D @ x_eps - b)    # still solves A x = b
    A = op_dense(D)
    res = oracle.ta_minnorm_bisect(A, b, x_eps, tol=1e-5, tol_normal=0.0, max_iter=400000)
    assert res.status == Status.OK and res.reason == Reason.GAP
    assert res.rho_lower <= nx * (1 + 1e-12)
    assert res.rho_upper - res.rho_lower <= 1e-5 * np.linalg.norm(x_eps)
    assert res.rel_res <= 1e-5 * (1 + 1e-9)
    assert np.linalg.norm(res.x) <= res.rho_upper * (1 + 1e-12)
    assert abs(np.linalg.norm(res.x) - nx) <= 2e-5 * nx
    assert np.linalg.norm(res.x - xs) <= 1e-2 * nx
    for rho, st, rs, hi, lo, it in res.trip_log:
        assert lo <= nx * (1 + 1e-12)


def test_ta_minnorm_hybrid_inconsistent_uses_normal_system():
    """Sec. 5.2: when CTA's x does not solve A x = b, TA runs on (AᵀA, Aᵀb)."""
    p = gen.dense_low_rank(12, 16, 5, seed=6)
    rng = np.random.default_rng(6)
    b = p.b + 0.5 * rng.standard_normal(12)
    res = oracle.ta_minnorm(op_dense(p.dense), b, tol=1e-4, tol_cta=1e-8, tol_normal=1e-9,
                            max_iter=200000)
    assert res.normal_system
    xs = minnorm(p.dense, b)
    assert res.status == Status.OK
    assert np.linalg.norm(res.x - xs) <= 1e-3 * np.linalg.norm(xs)


def test_ta_minnorm_hybrid_consistent():
    rng = np.random.default_rng(12)
    D = rng.standard_normal((5, 9))
    b = D @ rng.standard_normal(9)
    res = oracle.ta_minnorm(op_dense(D), b, tol=1e-4, tol_cta=1e-10, tol_normal=0.0,
                            max_iter=300000)
    assert not res.normal_system and res.status == Status.OK
    xs = minnorm(D, b)
    assert res.rho_lower <= np.linalg.norm(xs) * (1 + 1e-12)
    assert np.linalg.norm(res.x - xs) <= 1e-3 * np.linalg.norm(xs)


# --------------------------------------------------------------------------- TA for LP feasibility (Sec. 6)

def test_ta_lp_identity_golden():
    g = golden("ta_lp_identity.json")
    rhos = []
    res = oracle.ta_solve(op_dense(g["A"]), np.array(g["b"]), tol=1e-14, tol_normal=1e-14, max_iter=10,
                          nonneg=True, observer=lambda k, x, bp, rho, a: rhos.append(rho))
    assert rhos[0] == pytest.approx(g["rho_after_1"], rel=1e-15)
    assert res.iters == g["iters"] and res.reason == Reason.WITNESS     # Farkas: b_2 < 0
    np.testing.assert_allclose(res.x, g["x_final"], rtol=1e-14, atol=1e-14)


def test_ta_lp_feasible_keeps_nonnegative_iterates():
    """Sec. 6: with b = A x_+ for some x_+ >= 0 the c_+ iteration finds x >= 0 with
    ||Ax - b|| <= tol ||b||; every iterate is a convex combination of nonnegative
    vectors, so x' >= 0 throughout."""
    rng = np.random.default_rng(21)
    D = rng.uniform(0.0, 1.0, (8, 20))
    xp = rng.uniform(0.0, 1.0, 20)
    b = D @ xp
    neg = []
    res = oracle.ta_solve(op_dense(D), b, tol=1e-6, tol_normal=0.0, max_iter=200000, nonneg=True,
                          observer=lambda k, x, bp, rho, a: neg.append(x.min()))
    assert res.reason == Reason.RESIDUAL and res.rel_res <= 1e-6 * (1 + 1e-9)
    assert min(neg) >= 0.0 and res.x.min() >= 0.0


def test_ta_lp_infeasible_hits_rho_bound():
    """b with no nonnegative preimage: c_+ keeps an ascent direction along which rho grows
    without the residual closing; the termination bound on rho ends the test."""
    D = np.array([[1.0, 1.0], [1.0, 1.0 + 1e-3]])
    b = np.array([1.0, -1.0])                   # x = A^{-1} b has mixed signs
    res = oracle.ta_solve(op_dense(D), b, tol=1e-9, tol_normal=1e-12, max_iter=100000, nonneg=True,
                          rho_max=1e6)
    assert res.reason in (Reason.RHO_BOUND, Reason.WITNESS)
    assert res.x.min() >= 0.0 and res.rel_res > 1e-3


# ------------------------------------------------------------------ enhanced CTA (Sec. 3.2)

def test_enhanced_stop_closed_form_scaled_orthogonal():
    """A = 2Q (Q orthogonal): H = 4I, so one first-order step annihilates the residual
    (alpha_{1,1} = 1/4) and the enhanced algorithm stops at j = 1 with x^ = A^{-1} b."""
    import oracle.cta as ocx
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((16, 16)))
    A = 2.0 * Q
    b = rng.standard_normal(16)
    p = gen.Problem(name="q", m=16, n=16, fmt="dense", dense=A, b=b)
    res = ocx.cta_solve(oracle.make_operator(p), b, tol=1e-30, tol_normal=1e-8, max_iter=5, t_max=2,
                        cycle=ocx.FIXED, enhanced=True)
    assert res.reason == oracle.Reason.ENHANCED and res.iters == 1
    np.testing.assert_allclose(res.x, Q.T @ b / 2.0, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_enhanced_stop_is_repeated_first_order_steps(seed):
    """Wherever the enhanced stop fires, x^ equals j applications of F_1 (the order-1
    step of the plain iteration, Eq. eqcoeff with t = 1) from the same state, b - A x^ equals
    the returned residual, the returned residual meets the test, and no smaller j does."""
    import oracle.cta as ocx
    rng = np.random.default_rng(seed)
    m, n = 30, 45
    A = rng.standard_normal((m, 6)) @ rng.standard_normal((6, n)) + 0.05 * rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n)
    p = gen.Problem(name="e", m=m, n=n, fmt="dense", dense=A, b=b)
    op = oracle.make_operator(p)
    thr = (1e-3 * np.linalg.norm(A.T @ b)) ** 2
    hit, k = None, 0
    x, r = np.zeros(n), b.copy()
    while hit is None and k < 200:
        hit = ocx.enhanced_stop(op, x, r, 4, thr)
        if hit is None:
            x, r, _, _, _ = ocx.cta_step(op, x, r, 5)
            k += 1
    assert hit is not None
    xh, rh, j = hit
    xs, rs = x.copy(), r.copy()
    for _ in range(j):
        xs, rs, _, _, _ = ocx.cta_step(op, xs, rs, 1)
    np.testing.assert_allclose(xh, xs, rtol=1e-9, atol=1e-12 * np.linalg.norm(xs))
    assert np.linalg.norm((b - A @ xh) - rh) <= 1e-9 * np.linalg.norm(b)
    assert np.linalg.norm(A.T @ rh) ** 2 <= thr
    assert j == 1 or ocx.enhanced_stop(op, x, r, j - 1, thr) is None
