"""The products A x and Aᵀ y of every SpMV variant against scipy (needs a GB300).

The plan picks its kernel from the operator's structure: few short runs of x per
row tile (stencils) -> run-staged tiles; banded but with more runs, or more staged
entries than a stage holds -> x-window tiles; unstructured short rows -> generic
tiles; long rows -> warp per row. Each structure below lands on one of them; every
entry of the product must sit within the FP64 dot-product error bound
k u (|A| |x|)_i of scipy's value, k the row length.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def banded(n, offsets, seed):
    """n x n with the given diagonals, N(0,1) values, diagonal shifted for conditioning."""
    rng = np.random.default_rng(seed)
    diags = [rng.standard_normal(n - abs(o)) for o in offsets]
    S = sp.diags(diags, offsets, shape=(n, n), format="csr")
    S = (S + sp.identity(n) * 8.0).tocsr()
    S.sort_indices()
    return S


def banded_with_empty_rows(n, seed):
    """Tridiagonal-plus-far-band matrix with every 7th row and a block of 300 rows emptied."""
    S = banded(n, [-700, -1, 0, 1, 700], seed).tolil()
    for i in list(range(0, n, 7)) + list(range(10000, 10300)):
        S.rows[i] = []
        S.data[i] = []
    return S.tocsr()


def from_scipy(S, seed=0):
    rng = np.random.default_rng(seed + 100)
    S = S.tocsr()
    S.sort_indices()
    return gen.Problem(name="custom", m=S.shape[0], n=S.shape[1], fmt="csr", dense=None,
                       rowptr=S.indptr.astype(np.int32), colidx=S.indices.astype(np.int32),
                       vals=S.data.astype(np.float64), b=rng.standard_normal(S.shape[0]),
                       x_known=None, meta={})


STRUCTURES = {
    # three runs per 256-row tile (rows below, at and above): run-staged
    "stencil_300": lambda: gen.convdiff_stencil(300),
    # one merged run per tile: run-staged
    "stencil_40": lambda: gen.convdiff_stencil(40),
    "clement_5001": lambda: gen.clement(5001),
    # five diagonals 500 apart: banded (window 2256), up to five runs -> x-window tiles
    "five_runs": lambda: from_scipy(banded(20000, [-1000, -500, 0, 500, 1000], 1)),
    # four runs of 256 entries: more than a run stage holds -> x-window tiles
    "wide_runs": lambda: from_scipy(banded(20000, [-900, -300, 300, 900], 2)),
    # rectangular banded (m != n; Aᵀ run-staged too)
    "rect_banded": lambda: from_scipy(sp.diags([np.random.default_rng(5).standard_normal(20000)] * 3, [0, 700, 1500],
                                               shape=(20000, 22000), format="csr")),
    # banded with empty rows inside tiles
    "holes": lambda: from_scipy(banded_with_empty_rows(30000, 7)),
    # unstructured short rows -> generic tiles
    "random_short": lambda: gen.random_csr(30000, 20000, density=6 / 20000, seed=3),
    # long rows -> warp per row
    "random_long": lambda: gen.random_csr(2000, 50000, density=300 / 50000, seed=4),
}


def check_product(S, x, y):
    ref = S @ x
    k = np.maximum(np.diff(S.indptr), 1)
    bound = 1.01 * k * U * (abs(S) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= bound), float(np.max(np.abs(y - ref) / bound))


@pytest.mark.parametrize("name", sorted(STRUCTURES))
def test_products_match_scipy(tacta, name):
    import torch
    p = STRUCTURES[name]()
    S = p.scipy()
    d = torch.device("cuda:0")
    A = tacta.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n))
    plan = tacta.Plan(A)
    rng = np.random.default_rng(7)
    for trial in range(2):
        x = rng.standard_normal(p.n)
        y = plan.matvec(torch.from_numpy(x).to(d)).cpu().numpy()
        check_product(S, x, y)
        w = rng.standard_normal(p.m)
        z = plan.matvec(torch.from_numpy(w).to(d), transpose=True).cpu().numpy()
        check_product(S.T.tocsr(), w, z)
    plan.close()


@pytest.mark.parametrize("name", ["five_runs", "wide_runs", "stencil_300", "rect_banded", "holes"])
def test_cta_trajectory_per_variant(tacta, name):
    """Four CTA steps (t = 1..4, 20 products) against the oracle on each banded variant."""
    import torch
    p = STRUCTURES[name]()
    d = torch.device("cuda:0")
    A = tacta.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n))
    b = torch.from_numpy(np.ascontiguousarray(p.b)).to(d)
    x, hist, info = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=4)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=4)
    assert info["iters"] == ref.iters and info["matvecs"] == ref.matvecs
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-8)


@pytest.mark.parametrize("kind", ["csr", "dense"])
@pytest.mark.parametrize("transpose", [False, True])
def test_plan_residual(kind, transpose):
    """tacta_plan_residual: b - A x and b - Aᵀ x through the product kernels' residual
    epilogue, entry by entry against the host's FP64 within k u (|b| + |A||x|)."""
    import torch
    import paper_2304_12168_gb300 as tacta
    tacta.load_library()
    rng = np.random.default_rng(21)
    m, n = 300, 170
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < (0.08 if kind == "csr" else 1.0))
    S = sp.csr_matrix(D)
    dev = torch.device("cuda:0")
    if kind == "csr":
        A = tacta.CSR(torch.from_numpy(S.indptr.astype(np.int32)).to(dev), torch.from_numpy(S.indices.astype(np.int32)).to(dev),
                      torch.from_numpy(S.data).to(dev), (m, n))
    else:
        A = torch.from_numpy(D).to(dev)
    plan = tacta.Plan(A)
    M = D.T if transpose else D
    x = rng.standard_normal(M.shape[1])
    b = rng.standard_normal(M.shape[0])
    r = plan.residual(torch.from_numpy(x).to(dev), torch.from_numpy(b).to(dev), transpose=transpose).cpu().numpy()
    plan.close()
    ref = b - M @ x
    bound = (M.shape[1] + 1) * 2.0 ** -53 * (np.abs(b) + np.abs(M) @ np.abs(x))
    assert np.all(np.abs(r - ref) <= bound)
