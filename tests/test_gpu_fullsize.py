"""Full-size workloads against the FP64 oracle (needs a GB300).

At full size the oracle runs only a few steps in seconds, so these tests compare
fixed-length trajectories (the same launch configuration the benchmark times:
plan, tiled kernels, captured graphs) and single steps from oracle states; runs
to tolerance are checked through properties that hold at any size (true residual
computed on the host, agreement of the FP32 refinement path with the FP64 one).
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

X_TOL = 1e-9


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def dev(p):
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    return (t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n)),
            torch.from_numpy(np.ascontiguousarray(p.b)).to(d))


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def stencil():
    return gen.convdiff_stencil(1000)


@pytest.fixture(scope="module")
def rect():
    return gen.lp_rect()


def test_stencil_1000_fixed_period(tacta, stencil):
    """The climb t = 1..4 (4 F_t steps, 20 products) on the 1e6-unknown stencil to 1e-9;
    the full period (8 steps) against the oracle's own spread under 1e-16 perturbations
    of b -- at this size the t = 5 solve amplifies rounding to ~1e-9 of x."""
    p = stencil
    A, b = dev(p)
    plan = tacta.Plan(A)
    Ao = oracle.make_operator(p)
    x, hist, info = plan.cta(b, tol=1e-30, tol_normal=0.0, max_iter=4)
    ref = oracle.cta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=4)
    assert info["iters"] == ref.iters == 4 and info["matvecs"] == ref.matvecs
    assert relerr(x.cpu().numpy(), ref.x) <= X_TOL
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-8)
    x, hist, info = plan.cta(b, tol=1e-30, tol_normal=0.0, max_iter=8)
    ref = oracle.cta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=8)
    rng = np.random.default_rng(11)
    bp = p.b * (1 + 1e-16 * rng.standard_normal(p.m))
    refp = oracle.cta_solve(Ao, bp, tol=1e-30, tol_normal=0.0, max_iter=8)
    spread = relerr(refp.x, ref.x)
    assert relerr(x.cpu().numpy(), ref.x) <= max(X_TOL, 10 * spread)
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-7)
    assert abs(info["rel_res"] - ref.rel_res) <= max(1e-10, 10 * abs(refp.rel_res - ref.rel_res))
    plan.close()


def test_stencil_1000_single_t5_step_mid_trajectory(tacta, stencil):
    import torch
    p = stencil
    Ao = oracle.make_operator(p)
    xk = oracle.cta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=5).x
    A, b = dev(p)
    x, hist, _ = tacta.cta_solve(A, b, torch.from_numpy(xk).to("cuda:0"), tol=1e-30, tol_normal=0.0,
                                 max_iter=1, t_max=5, cycle=2)
    ref = oracle.cta_solve(Ao, p.b, xk, tol=1e-30, tol_normal=0.0, max_iter=1, t_max=5, cycle=2)
    dx = np.linalg.norm(x.cpu().numpy() - ref.x)
    assert dx <= X_TOL * np.linalg.norm(ref.x - xk) + 1e-14 * np.linalg.norm(xk)
    assert float(hist[1]) == pytest.approx(ref.hist[1], rel=1e-9)


def test_clement_100001_fixed(tacta):
    p = gen.clement(100001)
    A, b = dev(p)
    x, hist, info = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=40)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=40)
    assert relerr(x.cpu().numpy(), ref.x) <= X_TOL
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-8)


def test_rect_lp_fixed_cta_and_ta(tacta, rect):
    """10,000 x 1,000,000 LP-like matrix, 31.6M nonzeros: CTA and TA trajectories."""
    p = rect
    A, b = dev(p)
    plan = tacta.Plan(A)
    Ao = oracle.make_operator(p)
    x, hist, info = plan.cta(b, tol=1e-30, tol_normal=0.0, max_iter=4)
    ref = oracle.cta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=4)
    assert relerr(x.cpu().numpy(), ref.x) <= X_TOL
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-8)
    x, hist, info = plan.ta(b, tol=1e-30, tol_normal=0.0, max_iter=4)
    ref = oracle.ta_solve(Ao, p.b, tol=1e-30, tol_normal=0.0, max_iter=4)
    assert relerr(x.cpu().numpy(), ref.x) <= X_TOL
    assert info["rho"] == pytest.approx(ref.rho, rel=1e-12)
    plan.close()


def test_rect_lp_to_1e8_fp64_and_mixed(tacta, rect):
    """Both precisions reach 1e-8 (true residual checked on the host with scipy) and
    their solutions agree; the mixed path's distance to the FP64 one is the stated
    error of the FP32 chain (components outside range(Aᵀ) that no residual sees)."""
    p = rect
    A, b = dev(p)
    plan = tacta.Plan(A)
    S = p.scipy()
    bn = np.linalg.norm(p.b)
    x64, _, i64 = plan.cta(b, tol=1e-8, tol_normal=0.0, max_iter=2000)
    x32, _, i32 = plan.cta(b, tol=1e-8, tol_normal=0.0, max_iter=2000, precision=tacta.PRECISION_MIXED)
    for x, info in ((x64, i64), (x32, i32)):
        xh = x.cpu().numpy()
        assert info["reason_name"] == "RESIDUAL"
        assert np.linalg.norm(p.b - S @ xh) / bn <= 1e-8 * (1 + 1e-6)
    assert relerr(x32.cpu().numpy(), x64.cpu().numpy()) <= 1e-6
    plan.close()


def test_rect_small_min_norm(tacta):
    """A scaled-down copy of the LP-like family (500 x 20000): the converged CTA solution
    is the minimum-norm one (dense pseudo-inverse on the host)."""
    p = gen.lp_rect(m=500, n=20000, per_col=8, dup_rows=25, x_density=0.05, seed=5)
    A, b = dev(p)
    x, _, info = tacta.cta_solve(A, b, tol=1e-12, tol_normal=0.0, max_iter=20000)
    xs = np.linalg.pinv(p.to_dense(), rcond=1e-10) @ p.b
    assert info["reason_name"] == "RESIDUAL"
    assert relerr(x.cpu().numpy(), xs) <= 1e-9
