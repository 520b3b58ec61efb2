"""Differentiable solve (torch.autograd.Function around CTA with adjoint solves),
checked against dense pseudo-inverse gradients and central finite differences
(needs a GB300)."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

TOL = dict(tol=1e-13, tol_normal=0.0, max_iter=200000)


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def _loss(x, xt):
    return ((x - xt) ** 2).sum()


def _square(seed, n=64):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.linspace(1.0, 3.0, n)) @ P.T, rng.standard_normal(n), rng.standard_normal(n)


def test_square_dense_gradient_matches_formula_and_fd(tacta):
    """64 x 64 nonsingular: dL/db = A^{-T} g, dL/dA = -A^{-T} g xᵀ (numpy, independent), and
    central differences (h = 1e-6) of L through the GPU forward."""
    import torch
    from paper_2304_12168_gb300.autograd import cta_solve_autograd
    D, b, xt = _square(1)
    A = torch.tensor(D, device="cuda:0", requires_grad=True)
    bt = torch.tensor(b, device="cuda:0", requires_grad=True)
    xtt = torch.tensor(xt, device="cuda:0")
    x = cta_solve_autograd(A, bt, **TOL)
    L = _loss(x, xtt)
    L.backward()
    xs = np.linalg.solve(D, b)
    g = 2 * (xs - xt)
    lam = np.linalg.solve(D.T, g)
    np.testing.assert_allclose(x.detach().cpu().numpy(), xs, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(bt.grad.cpu().numpy(), lam, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(A.grad.cpu().numpy(), -np.outer(lam, xs), rtol=1e-9, atol=1e-10)
    # central differences through the GPU forward on a few entries
    h = 1e-6
    rng = np.random.default_rng(0)
    for (i, j) in rng.integers(0, 64, size=(4, 2)):
        Dp, Dm = D.copy(), D.copy()
        Dp[i, j] += h
        Dm[i, j] -= h
        Lp = _loss(cta_solve_autograd(torch.tensor(Dp, device="cuda:0"), bt.detach(), **TOL), xtt).item()
        Lm = _loss(cta_solve_autograd(torch.tensor(Dm, device="cuda:0"), bt.detach(), **TOL), xtt).item()
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(A.grad[i, j].item(), rel=1e-5, abs=1e-7)


def test_min_norm_dense_gradient_matches_pinv_fd(tacta):
    """Full row rank 20 x 50: x = A⁺ b. The gradient is checked against central differences
    of the dense pseudo-inverse solution (numpy, independent of the library)."""
    import torch
    from paper_2304_12168_gb300.autograd import cta_solve_autograd
    rng = np.random.default_rng(3)
    D = rng.standard_normal((20, 50))
    b = rng.standard_normal(20)
    xt = rng.standard_normal(50)
    A = torch.tensor(D, device="cuda:0", requires_grad=True)
    bt = torch.tensor(b, device="cuda:0", requires_grad=True)
    x = cta_solve_autograd(A, bt, **TOL)
    _loss(x, torch.tensor(xt, device="cuda:0")).backward()

    def L(Dv, bv):
        return float(np.sum((np.linalg.pinv(Dv) @ bv - xt) ** 2))
    h = 1e-6
    for (i, j) in rng.integers(0, [20, 50], size=(5, 2)):
        Dp, Dm = D.copy(), D.copy()
        Dp[i, j] += h
        Dm[i, j] -= h
        assert (L(Dp, b) - L(Dm, b)) / (2 * h) == pytest.approx(A.grad[i, j].item(), rel=1e-5, abs=1e-8)
    for i in rng.integers(0, 20, size=3):
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        assert (L(D, bp) - L(D, bm)) / (2 * h) == pytest.approx(bt.grad[i].item(), rel=1e-5, abs=1e-8)


def test_csr_gradient_on_pattern(tacta):
    """Stencil 12 x 12 in CSR: dL/dvals is the dense gradient -lambda xᵀ read on the pattern."""
    import torch
    import paper_2304_12168_gb300 as t
    from paper_2304_12168_gb300.autograd import cta_solve_autograd
    p = gen.convdiff_stencil(12)
    d = "cuda:0"
    vals = torch.tensor(p.vals, device=d, requires_grad=True)
    A = t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d), vals, (p.m, p.n))
    bt = torch.tensor(p.b, device=d, requires_grad=True)
    xt = np.random.default_rng(2).standard_normal(p.n)
    x = cta_solve_autograd(A, bt, **TOL)
    _loss(x, torch.tensor(xt, device=d)).backward()
    Dn = p.to_dense()
    xs = np.linalg.solve(Dn, p.b)
    lam = np.linalg.solve(Dn.T, 2 * (xs - xt))
    rows = np.repeat(np.arange(p.m), np.diff(p.rowptr))
    np.testing.assert_allclose(vals.grad.cpu().numpy(), -lam[rows] * xs[p.colidx], rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(bt.grad.cpu().numpy(), lam, rtol=1e-8, atol=1e-10)


def test_min_norm_2000x8000_gradient(tacta):
    """Dense full-row-rank 2000 x 8000 N(0,1) (the differentiable workload): gradients against
    the closed form with (A Aᵀ)^{-1} from numpy, and a directional central difference in b."""
    import torch
    from paper_2304_12168_gb300.autograd import cta_solve_autograd
    rng = np.random.default_rng(5)
    D = rng.standard_normal((2000, 8000))
    b = rng.standard_normal(2000)
    xt = rng.standard_normal(8000)
    A = torch.tensor(D, device="cuda:0", requires_grad=True)
    bt = torch.tensor(b, device="cuda:0", requires_grad=True)
    xtt = torch.tensor(xt, device="cuda:0")
    opts = dict(tol=1e-12, tol_normal=0.0, max_iter=20000)
    x = cta_solve_autograd(A, bt, **opts)
    _loss(x, xtt).backward()
    G = D @ D.T
    w = np.linalg.solve(G, b)
    xs = D.T @ w
    g = 2 * (xs - xt)
    lam = np.linalg.solve(G, D @ g)
    np.testing.assert_allclose(bt.grad.cpu().numpy(), lam, rtol=1e-7, atol=1e-9)
    gA = np.outer(w, g - D.T @ lam) - np.outer(lam, xs)
    assert np.linalg.norm(A.grad.cpu().numpy() - gA) <= 1e-7 * np.linalg.norm(gA)
    v = rng.standard_normal(2000)
    h = 1e-6
    Lp = _loss(cta_solve_autograd(A.detach(), bt.detach() + h * torch.tensor(v, device="cuda:0"), **opts), xtt)
    Lm = _loss(cta_solve_autograd(A.detach(), bt.detach() - h * torch.tensor(v, device="cuda:0"), **opts), xtt)
    fd = (Lp - Lm).item() / (2 * h)
    assert fd == pytest.approx(float(bt.grad.cpu().numpy() @ v), rel=1e-5)


def test_stencil_256_forward_and_adjoint_trajectories(tacta):
    """The 256 x 256 stencil (n = 65,536) of the differentiable workload. CTA needs far more
    than a test's worth of iterations to converge there, so the forward and the adjoint
    solve run eight steps each and are compared with the oracle's eight-step trajectories
    on A and Aᵀ; the pattern gradient must equal -lambda[row] x[col] exactly."""
    import torch
    import paper_2304_12168_gb300 as t
    from paper_2304_12168_gb300.autograd import cta_solve_autograd
    p = gen.convdiff_stencil(256)
    d = "cuda:0"
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=8)
    vals = torch.tensor(p.vals, device=d, requires_grad=True)
    A = t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d), vals, (p.m, p.n))
    bt = torch.tensor(p.b, device=d, requires_grad=True)
    xt = np.random.default_rng(4).standard_normal(p.n)
    x = cta_solve_autograd(A, bt, **opts)
    _loss(x, torch.tensor(xt, device=d)).backward()
    import oracle
    S = p.scipy()
    Ao = oracle.make_operator(p)
    ref = oracle.cta_solve(Ao, p.b, **opts)
    xs = x.detach().cpu().numpy()
    assert np.linalg.norm(xs - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    ST = S.T.tocsr()
    pt = gen.Problem(name="stencil_T", m=p.n, n=p.m, fmt="csr", rowptr=ST.indptr.astype(np.int32),
                     colidx=ST.indices.astype(np.int32), vals=ST.data.astype(np.float64),
                     b=2 * (xs - xt))
    lam_ref = oracle.cta_solve(oracle.make_operator(pt), pt.b, **opts).x
    lam = bt.grad.cpu().numpy()
    assert np.linalg.norm(lam - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    rows = np.repeat(np.arange(p.m), np.diff(p.rowptr))
    np.testing.assert_array_equal(vals.grad.cpu().numpy(), -lam[rows] * xs[p.colidx])
