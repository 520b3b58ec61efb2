"""GPU solvers against the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (FP64 path): relative solution error <= 1e-9 and final true
relative residual equal within 1e-10. Fixed-length runs must take the same
number of steps with the same residual history; runs to a tolerance must stop
inside the window the oracle's own stop index spans under 1e-16 perturbations
of b (tests/oracle_spread.py: 16 perturbed runs, Tukey's fences, +-1 step),
which is the unperturbed index +-1 whenever the oracle's index does not move.
"""
import numpy as np
import pytest

import gen
import oracle
from oracle import Reason
from tests.oracle_spread import stop_index_window

pytestmark = pytest.mark.gpu

X_TOL = 1e-9
RES_TOL = 1e-10

# How parity is judged. CTA's auxiliary solve of order t amplifies rounding
# differences in the moments phi_i by up to the condition number of the Hankel
# matrix, so two correct FP64 implementations that sum in different orders
# follow trajectories that agree to ~1e-12 for tens of steps and then drift
# apart (both still converge to the same solution). The tests therefore
# compare (1) single F_t steps and TA steps taken from the same state, (2)
# short fixed-length trajectories, and (3) converged solutions.

REASON = {int(Reason.RESIDUAL): "RESIDUAL", int(Reason.NORMAL): "NORMAL",
          int(Reason.MAXITER): "MAXITER", int(Reason.ZERO_RHS): "ZERO_RHS",
          int(Reason.GAP): "GAP", int(Reason.BREAKDOWN): "BREAKDOWN",
          int(Reason.WITNESS): "WITNESS", int(Reason.RHO_BOUND): "RHO_BOUND"}


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()          # a missing library is an error here, not a skip
    torch.cuda.set_device(0)
    return t


def dev(p):
    """gen.Problem -> (matrix argument, b) as CUDA tensors."""
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    b = torch.from_numpy(np.ascontiguousarray(p.b)).to(d)
    if p.fmt == "dense":
        return torch.from_numpy(np.ascontiguousarray(p.dense)).to(d), b
    return t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                 torch.from_numpy(p.vals).to(d), (p.m, p.n)), b


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def check_iters(got, solve_name, p, x0, okw):
    """The GPU's stop index lies in the oracle's own rounding window (stop_index_window)."""
    lo, hi, its = stop_index_window(solve_name, p, x0, okw)
    assert lo <= got <= hi, (got, lo, hi, sorted(its.tolist()))


def check_cta(tacta, p, x0=None, iter_slack=None, **kw):
    A, b = dev(p)
    import torch
    x0d = None if x0 is None else torch.from_numpy(x0).to("cuda:0")
    x, hist, info = tacta.cta_solve(A, b, x0d, **kw)
    okw = {k: v for k, v in kw.items() if k in ("tol", "tol_normal", "max_iter", "t_max", "cycle",
                                                 "recompute_every", "pivot_tol")}
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, x0, **okw)
    xg = x.cpu().numpy()
    if iter_slack is None:       # run to tolerance: the stop index is rounding-sensitive
        check_iters(info["iters"], "cta_solve", p, x0, okw)
        assert info["reason_name"] == REASON[int(ref.reason)]
    else:
        assert abs(info["iters"] - ref.iters) <= iter_slack, (info, ref.iters, ref.reason)
    if info["iters"] == ref.iters:
        assert info["reason_name"] == REASON[int(ref.reason)]
        assert info["matvecs"] == ref.matvecs
        h = hist.cpu().numpy()
        assert h.size == len(ref.hist)
        if iter_slack == 0:      # fixed-length trajectory: the whole history agrees
            np.testing.assert_allclose(h, ref.hist, rtol=1e-8, atol=1e-13)
    assert relerr(xg, ref.x) <= X_TOL, relerr(xg, ref.x)
    assert abs(info["rel_res"] - ref.rel_res) <= RES_TOL
    return xg, info, ref


# ------------------------------------------------------------------ CTA

@pytest.mark.parametrize("N", [7, 50])
def test_cta_stencil_to_tolerance(tacta, N):
    """Stencil of 49 rows (one block) and 2500 rows (ten blocks + ragged tail)."""
    p = gen.convdiff_stencil(N)
    xg, info, ref = check_cta(tacta, p, tol=1e-12, tol_normal=0.0, max_iter=20000)
    assert info["reason_name"] == "RESIDUAL"
    assert np.abs(xg - 1.0).max() < 1e-8


def test_cta_stencil_fixed_iterations(tacta):
    p = gen.convdiff_stencil(64)
    check_cta(tacta, p, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=64)


@pytest.mark.parametrize("t", [1, 2, 3, 4, 5])
def test_cta_single_step_from_oracle_states(tacta, t):
    """One F_t from the same state x_k at several points of the oracle's trajectory:
    the step x_{k+1} - x_k and the new residual agree to 1e-9 relative."""
    import torch
    p = gen.convdiff_stencil(50)
    Ao = oracle.make_operator(p)
    A, b = dev(p)
    for k in (0, 30, 120):
        xk = oracle.cta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=k).x if k else np.zeros(p.n)
        x, hist, info = tacta.cta_solve(A, b, torch.from_numpy(xk).to("cuda:0"), tol=1e-30,
                                        tol_normal=0.0, max_iter=1, t_max=t, cycle=2)
        ref = oracle.cta_solve(Ao, p.b, xk, tol=1e-30, tol_normal=0.0, max_iter=1, t_max=t, cycle=2)
        # the order-t auxiliary solve amplifies rounding late in the trajectory: the
        # moments summed in another order differ by ~sqrt(n) u relative, so the oracle's
        # own spread under a perturbation of x_k of that size bounds what any summation
        # order can reproduce
        eps = np.sqrt(p.n) * 2.0 ** -53
        xp = xk * (1 + eps * np.random.default_rng(k + t).standard_normal(p.n))
        refp = oracle.cta_solve(Ao, p.b, xp, tol=1e-30, tol_normal=0.0, max_iter=1, t_max=t, cycle=2)
        spread = np.linalg.norm((refp.x - xp) - (ref.x - xk))
        # x'' - x' loses digits to cancellation once the step is small next to x':
        # judge the step to 1e-9 of itself (or the spread) plus rounding of ||x'||
        step_o = ref.x - xk
        dx = np.linalg.norm(x.cpu().numpy() - ref.x)
        assert dx <= max(X_TOL * np.linalg.norm(step_o), 10 * spread) + 1e-14 * np.linalg.norm(xk), (k, dx, spread)
        assert hist.cpu().numpy()[1] == pytest.approx(ref.hist[1], rel=1e-9)


@pytest.mark.parametrize("n", [101, 1001])
def test_cta_clement_singular(tacta, n):
    p = gen.clement(n)
    xg, info, ref = check_cta(tacta, p, tol=1e-11, tol_normal=0.0, max_iter=50000)
    assert info["reason_name"] == "RESIDUAL"


def test_cta_dense_gaussian_fixed(tacta):
    p = gen.dense_gaussian(256, 256, seed=0)
    check_cta(tacta, p, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=40)


def test_cta_dense_low_rank_minnorm(tacta):
    p = gen.dense_low_rank(256, 256, 128, seed=1)
    xg, info, ref = check_cta(tacta, p, tol=1e-10, tol_normal=0.0, max_iter=20000)
    xs = np.linalg.pinv(p.dense, rcond=1e-10) @ p.b
    assert relerr(xg, xs) < 1e-7


def test_cta_dense_rectangular_both_kernels(tacta):
    """Wide (n >= 64: warp-per-row A) and tall-thin (m < 64: thread-per-row Aᵀ) dense shapes."""
    rng = np.random.default_rng(5)
    for m, n in ((40, 300), (300, 40)):
        D = rng.standard_normal((m, n))
        b = D @ rng.standard_normal(n)
        p = gen.Problem(f"d{m}x{n}", m, n, "dense", np.ascontiguousarray(D), b=b)
        check_cta(tacta, p, tol=1e-11, tol_normal=0.0, max_iter=5000)


def test_cta_ragged_csr_long_and_empty_rows(tacta):
    p = gen.random_csr(700, 300, density=0.02, seed=7, empty_rows=30, long_rows=5, long_len=250)
    check_cta(tacta, p, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=24)
    check_cta(tacta, p, tol=1e-10, tol_normal=1e-10, max_iter=20000)
    p2 = gen.random_csr(300, 5000, density=0.03, seed=8, empty_rows=3)     # long rows: warp kernel
    check_cta(tacta, p2, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=24)
    check_cta(tacta, p2, tol=1e-11, tol_normal=0.0, max_iter=20000)


def test_cta_inconsistent_normal_stop(tacta):
    p = gen.dense_low_rank(60, 60, 20, seed=4)
    rng = np.random.default_rng(4)
    p.b = p.b + rng.standard_normal(60)
    xg, info, ref = check_cta(tacta, p, tol=1e-12, tol_normal=1e-11, max_iter=20000)
    assert info["reason_name"] == "NORMAL"


@pytest.mark.parametrize("t_max,cycle", [(1, 0), (3, 1), (5, 2)])
def test_cta_orders_and_cycles(tacta, t_max, cycle):
    p = gen.convdiff_stencil(20)
    check_cta(tacta, p, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=24, t_max=t_max, cycle=cycle)


@pytest.mark.parametrize("t", [6, 7, 8])
def test_cta_high_orders_single_step(tacta, t):
    """Orders beyond the paper's cycle (t <= 8 supported): one F_t from the same state.
    Their moments span 2t powers of H and the scaled Hankel matrix is so ill-conditioned
    that the oracle itself moves by ~1e-8..1e-7 of the step when b is perturbed by 1e-16.
    The new residual norm (the quantity F_t minimises) must still agree to 1e-9, and the
    GPU's step must sit within 10x the oracle's own perturbation spread."""
    import torch
    p = gen.convdiff_stencil(20)
    Ao = oracle.make_operator(p)
    A, b = dev(p)
    xk = oracle.cta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=10).x
    x, hist, info = tacta.cta_solve(A, b, torch.from_numpy(xk).to("cuda:0"), tol=1e-30,
                                    tol_normal=0.0, max_iter=1, t_max=t, cycle=2)
    kw = dict(tol=1e-30, tol_normal=0.0, max_iter=1, t_max=t, cycle=2)
    ref = oracle.cta_solve(Ao, p.b, xk, **kw)
    rng = np.random.default_rng(7)
    spread = max(np.linalg.norm(oracle.cta_solve(Ao, p.b * (1 + 1e-16 * rng.standard_normal(p.m)),
                                                 xk, **kw).x - ref.x) for _ in range(3))
    dx = np.linalg.norm(x.cpu().numpy() - ref.x)
    assert dx <= 10 * spread + X_TOL * np.linalg.norm(ref.x - xk), (dx, spread)
    assert hist.cpu().numpy()[1] == pytest.approx(ref.hist[1], rel=1e-9)


def test_cta_warm_start_and_recompute_period(tacta):
    p = gen.convdiff_stencil(30)
    x0 = np.random.default_rng(1).standard_normal(p.n)
    check_cta(tacta, p, x0=x0, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=30, recompute_every=7)
    check_cta(tacta, p, x0=x0, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=30, recompute_every=0)


def test_cta_graph_and_stream_paths_agree_bitwise(tacta):
    p = gen.convdiff_stencil(40)
    A, b = dev(p)
    x1, h1, i1 = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=77, use_graph=1)
    x2, h2, i2 = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=77, use_graph=0,
                                 poll_every=5)
    assert i1["iters"] == i2["iters"] == 77
    assert (x1 == x2).all() and (h1 == h2).all()


def test_cta_plan_reuse_many_rhs(tacta):
    import torch
    p = gen.convdiff_stencil(16)
    A, _ = dev(p)
    plan = tacta.Plan(A)
    rng = np.random.default_rng(2)
    for j in range(3):
        bj = rng.standard_normal(p.m)
        x, _, info = plan.cta(torch.from_numpy(bj).to("cuda:0"), tol=1e-12, tol_normal=0.0, max_iter=5000)
        ref = oracle.cta_solve(oracle.make_operator(p), bj, tol=1e-12, tol_normal=0.0, max_iter=5000)
        assert relerr(x.cpu().numpy(), ref.x) <= X_TOL
    plan.close()


def test_cta_host_buffers(tacta):
    """on_device = 0: host arrays in, the library does the copies."""
    p = gen.convdiff_stencil(12)
    x, hist, info = tacta.cta_solve(p, p.b, tol=1e-30, tol_normal=0.0, max_iter=30)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=30)
    assert isinstance(x, np.ndarray) and isinstance(hist, np.ndarray)
    assert relerr(x, ref.x) <= X_TOL and info["iters"] == ref.iters == 30
    np.testing.assert_allclose(hist, ref.hist, rtol=1e-8)


# ------------------------------------------------------------------ TA

def check_ta(tacta, p, x0=None, iter_slack=None, x_tol=X_TOL, **kw):
    import torch
    A, b = dev(p)
    x0d = None if x0 is None else torch.from_numpy(x0).to("cuda:0")
    x, hist, info = tacta.ta_solve(A, b, x0d, **kw)
    okw = {k: v for k, v in kw.items() if k in ("tol", "tol_normal", "max_iter", "recompute_every")}
    ref = oracle.ta_solve(oracle.make_operator(p), p.b, x0, **okw)
    xg = x.cpu().numpy()
    if iter_slack is None:
        check_iters(info["iters"], "ta_solve", p, x0, okw)
    else:
        assert abs(info["iters"] - ref.iters) <= iter_slack, (info, ref.iters, ref.reason)
    assert relerr(xg, ref.x) <= x_tol, relerr(xg, ref.x)
    assert abs(info["rel_res"] - ref.rel_res) <= RES_TOL
    assert info["rho"] == pytest.approx(ref.rho, rel=1e-9)
    if iter_slack == 0:
        np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-8, atol=1e-13)
    return xg, info, ref


def test_ta_dense_consistent(tacta):
    """Underdetermined consistent system run to 1e-12: both land on A⁺b (x ∈ range(Aᵀ))."""
    p = gen.dense_gaussian(40, 60, seed=2)
    xg, info, ref = check_ta(tacta, p, tol=1e-12, tol_normal=0.0, max_iter=20000)
    xs = np.linalg.pinv(p.dense) @ p.b
    assert relerr(xg, xs) <= 1e-9


def test_ta_fixed_iterations(tacta):
    check_ta(tacta, gen.convdiff_stencil(30), iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=100)
    check_ta(tacta, gen.dense_gaussian(40, 60, seed=2), iter_slack=0, tol=1e-30, tol_normal=0.0,
             max_iter=20)


def test_ta_single_step_from_oracle_states(tacta):
    """One TA iteration from the same warm start (b' = A x0, rho = ||x0||)."""
    import torch
    p = gen.dense_gaussian(40, 60, seed=2)
    Ao = oracle.make_operator(p)
    A, b = dev(p)
    for k in (5, 60, 200):
        xk = oracle.ta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=k).x
        for steps in (1, 2):
            x, _, info = tacta.ta_solve(A, b, torch.from_numpy(xk).to("cuda:0"), tol=1e-30,
                                        tol_normal=0.0, max_iter=steps)
            ref = oracle.ta_solve(Ao, p.b, xk, tol=1e-30, tol_normal=0.0, max_iter=steps)
            assert info["rho"] == pytest.approx(ref.rho, rel=1e-12)
            dx = np.linalg.norm(x.cpu().numpy() - ref.x)
            assert dx <= X_TOL * np.linalg.norm(ref.x - xk) + 1e-14 * np.linalg.norm(xk), (k, steps, dx)


def test_ta_warm_start(tacta):
    p = gen.dense_gaussian(30, 50, seed=3)
    x0 = 0.5 * np.random.default_rng(3).standard_normal(50)
    check_ta(tacta, p, x0=x0, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=20)


def test_ta_csr_rectangular(tacta):
    p = gen.random_csr(200, 900, density=0.02, seed=11, empty_rows=0)
    check_ta(tacta, p, iter_slack=0, tol=1e-30, tol_normal=0.0, max_iter=30)


# ------------------------------------------------------------------ hybrid minimum norm

def check_minnorm(tacta, p, **kw):
    """Algorithm 2.5's outcome is judged by what Def. minnormapp fixes, not by the
    trip-by-trip path (TA's trajectory is as rounding-sensitive as CTA's): both
    sides bracket ||x_*|| within the gap, both answers meet the tolerance, and
    both are within the tolerance-implied distance of the minimum-norm solution."""
    A, b = dev(p)
    x, hist, info = tacta.ta_minnorm(A, b, **kw)
    okw = {k: v for k, v in kw.items() if k in ("tol", "tol_cta", "tol_normal", "max_iter")}
    ref = oracle.ta_minnorm(oracle.make_operator(p), p.b, **okw)
    xg = x.cpu().numpy()
    tol = kw["tol"]
    assert info["normal_system"] == int(ref.normal_system)
    assert info["reason_name"] == REASON[int(ref.reason)] == "GAP"
    D = p.to_dense()
    xs = np.linalg.pinv(D, rcond=1e-10) @ p.b
    nx = np.linalg.norm(xs)
    gap = tol * nx * 1.01
    for hi, lo in ((info["rho"], info["rho_lower"]), (ref.rho_upper, ref.rho_lower)):
        assert lo <= nx * (1 + 1e-9)                     # Cor. cor1 lower bound
        assert hi - lo <= 2 * gap + 1e-12                # gap closed
    assert abs(info["rho"] - ref.rho_upper) <= 2 * gap + 1e-12
    assert abs(info["rho_lower"] - ref.rho_lower) <= 2 * gap + 1e-12
    assert np.linalg.norm(xg) <= info["rho"] * (1 + 1e-12)
    assert relerr(xg, xs) <= 50 * tol and relerr(ref.x, xs) <= 50 * tol
    assert relerr(xg, ref.x) <= 100 * tol
    return x, info, ref


def test_minnorm_consistent(tacta):
    rng = np.random.default_rng(12)
    D = rng.standard_normal((5, 9))
    p = gen.Problem("mn5x9", 5, 9, "dense", np.ascontiguousarray(D), b=D @ rng.standard_normal(9))
    check_minnorm(tacta, p, tol=1e-4, tol_cta=1e-10, tol_normal=0.0, max_iter=300000)


def test_minnorm_inconsistent_normal_system(tacta):
    p = gen.dense_low_rank(12, 16, 5, seed=6)
    p.b = p.b + 0.5 * np.random.default_rng(6).standard_normal(12)
    check_minnorm(tacta, p, tol=1e-4, tol_cta=1e-8, tol_normal=1e-9, max_iter=200000)


# ------------------------------------------------------------------ edge cases

def test_zero_rhs(tacta):
    import torch
    p = gen.convdiff_stencil(9)
    A, _ = dev(p)
    z = torch.zeros(p.m, dtype=torch.float64, device="cuda:0")
    for fn in (tacta.cta_solve, tacta.ta_solve, tacta.ta_minnorm):
        x, _, info = fn(A, z, tol=1e-10)
        assert info["reason_name"] == "ZERO_RHS" and info["status"] == 0
        assert not x.any()


def test_max_iter_zero_and_tiny_shapes(tacta):
    p = gen.convdiff_stencil(5)
    xg, info, ref = check_cta(tacta, p, iter_slack=0, tol=1e-12, tol_normal=0.0, max_iter=0)
    assert info["iters"] == 0 and info["reason_name"] == "MAXITER"
    one = gen.Problem("1x1", 1, 1, "dense", np.array([[3.0]]), b=np.array([6.0]))
    xg, info, ref = check_cta(tacta, one, tol=1e-12, tol_normal=0.0, max_iter=10)
    assert xg[0] == pytest.approx(2.0, rel=1e-15)
    row = gen.Problem("1x7", 1, 7, "dense", np.arange(1.0, 8.0)[None, :], b=np.array([2.0]))
    check_cta(tacta, row, tol=1e-12, tol_normal=0.0, max_iter=10)


def test_all_zero_matrix(tacta):
    """nnz = 0: Aᵀb = 0, so x = 0 already solves the normal equation (Ex. exam1)."""
    p = gen.Problem("zero", 6, 4, "csr", None, np.zeros(7, np.int32), np.zeros(0, np.int32),
                    np.zeros(0), b=np.ones(6))
    xg, info, ref = check_cta(tacta, p, tol=1e-10, max_iter=10)
    assert info["reason_name"] == "NORMAL" and not xg.any()


def test_invalid_inputs_raise(tacta):
    import torch
    d = "cuda:0"
    b = torch.ones(3, dtype=torch.float64, device=d)
    bad = tacta.CSR(torch.tensor([0, 2, 1, 3], dtype=torch.int32, device=d),
                    torch.tensor([0, 1, 2], dtype=torch.int32, device=d),
                    torch.ones(3, dtype=torch.float64, device=d), (3, 3))
    with pytest.raises(tacta.TactaError, match="rowptr decreases"):
        tacta.cta_solve(bad, b)
    oob = tacta.CSR(torch.tensor([0, 1, 2, 3], dtype=torch.int32, device=d),
                    torch.tensor([0, 5, 2], dtype=torch.int32, device=d),
                    torch.ones(3, dtype=torch.float64, device=d), (3, 3))
    with pytest.raises(tacta.TactaError, match="out of range"):
        tacta.cta_solve(oob, b)
    p = gen.convdiff_stencil(4)
    A, bb = dev(p)
    with pytest.raises(tacta.TactaError, match="tol"):
        tacta.cta_solve(A, bb, tol=0.0)
    with pytest.raises(tacta.TactaError, match="t_max"):
        tacta.cta_solve(A, bb, t_max=9)


def test_nonfinite_input_reports_error(tacta):
    import torch
    p = gen.convdiff_stencil(6)
    A, b = dev(p)
    b[3] = float("nan")
    with pytest.raises(tacta.TactaError, match="NONFINITE"):
        tacta.cta_solve(A, b, tol=1e-10)


# ------------------------------------------------------------------ TA for LP feasibility (Sec. 6)

def test_ta_lp_identity_golden(tacta):
    """A = I, b = (3, -4): the c_+ iteration ends at the orthant projection (3, 0) with a
    Farkas certificate of infeasibility (golden fixture, hand-derived)."""
    import json
    import os
    import torch
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ta_lp_identity.json")))
    A = torch.tensor(g["A"], dtype=torch.float64, device="cuda:0")
    b = torch.tensor(g["b"], dtype=torch.float64, device="cuda:0")
    x, _, info = tacta.ta_solve(A, b, tol=1e-14, tol_normal=1e-14, max_iter=10, nonneg=1)
    assert info["status_name"] == "WITNESS" and info["iters"] == g["iters"]
    np.testing.assert_allclose(x.cpu().numpy(), g["x_final"], rtol=1e-14, atol=1e-14)


def _lp_problem(seed, fmt):
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.0, 1.0, (30, 80))
    D[rng.uniform(size=D.shape) < 0.6] = 0.0
    b = D @ rng.uniform(0.0, 1.0, 80)
    p = gen.Problem(f"lp{seed}", 30, 80, "dense", np.ascontiguousarray(D), b=b)
    return p.as_csr() if fmt == "csr" else p


@pytest.mark.parametrize("fmt", ["dense", "csr"])
def test_ta_lp_trajectory_and_feasible_solve(tacta, fmt):
    import torch
    p = _lp_problem(21, fmt)
    A, b = dev(p)
    Ao = oracle.make_operator(p)
    x, hist, info = tacta.ta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=25, nonneg=1)
    ref = oracle.ta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=25, nonneg=True)
    assert info["iters"] == ref.iters == 25
    assert relerr(x.cpu().numpy(), ref.x) <= X_TOL
    assert info["rho"] == pytest.approx(ref.rho, rel=1e-12)
    x, hist, info = tacta.ta_solve(A, b, tol=1e-6, tol_normal=0.0, max_iter=200000, nonneg=1)
    xg = x.cpu().numpy()
    assert info["reason_name"] == "RESIDUAL" and info["rel_res"] <= 1e-6
    assert xg.min() >= 0.0
    D = p.to_dense()
    assert np.linalg.norm(D @ xg - p.b) <= 1e-6 * np.linalg.norm(p.b) * (1 + 1e-9)


def test_ta_lp_rho_bound(tacta):
    import torch
    D = np.array([[1.0, 1.0], [1.0, 1.001]])
    A = torch.from_numpy(D).to("cuda:0")
    b = torch.tensor([1.0, -1.0], dtype=torch.float64, device="cuda:0")
    x, _, info = tacta.ta_solve(A, b, tol=1e-9, tol_normal=1e-12, max_iter=100000, nonneg=1, rho_max=1e6)
    ref = oracle.ta_solve(oracle.Operator(2, 2, "dense", dense=D), np.array([1.0, -1.0]), tol=1e-9,
                          tol_normal=1e-12, max_iter=100000, nonneg=True, rho_max=1e6)
    assert info["reason_name"] == REASON.get(int(ref.reason), ref.reason.name)
    assert x.cpu().numpy().min() >= 0.0
