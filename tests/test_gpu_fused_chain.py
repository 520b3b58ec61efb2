"""The fused CTA chain (all 2t products of a step in one cooperative launch) against the
oracle and against the one-launch-per-product path (needs a GB300).

Both paths compute every row of every product with the same arithmetic; only the
moments' partial sums are added in another fixed order. So fixed trajectories match
the oracle as the per-product path does, the two paths agree closely with each other,
and the fused path is deterministic (graph replay equals direct launches bit for bit).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def from_scipy(S, seed):
    S = sp.csr_matrix(S)
    S.sort_indices()
    rng = np.random.default_rng(seed)
    b = S @ rng.standard_normal(S.shape[1])
    return gen.Problem(name="s", m=S.shape[0], n=S.shape[1], fmt="csr",
                       rowptr=S.indptr.astype(np.int32), colidx=S.indices.astype(np.int32),
                       vals=S.data.astype(np.float64), b=b)


def rect_banded():
    """20000 x 22000, three diagonals at offsets 0, 700, 1500: A has 79 tiles, Aᵀ 86 (both
    ragged), so the grid is 86 blocks and some blocks have no tile of A."""
    rng = np.random.default_rng(11)
    return from_scipy(sp.diags([rng.standard_normal(20000)] * 3, [0, 700, 1500], shape=(20000, 22000)), 12)


CASES = {
    "stencil_24": lambda: gen.convdiff_stencil(24),      # 576 rows: 3 tiles, 3 blocks
    "stencil_300": lambda: gen.convdiff_stencil(300),    # 90000 rows: 352 tiles per product
    "rect_banded": rect_banded,
    "clement_5001": lambda: gen.clement(5001),
}


def dev(p):
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    return (t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n)),
            torch.from_numpy(np.ascontiguousarray(p.b)).to(d))


@pytest.mark.parametrize("name", list(CASES))
def test_fused_trajectory_matches_oracle(tacta, name):
    """40 F_t steps (ping-pong t = 1..5 and back) on the fused path: iterations, products,
    x (1e-9) and the residual history (1e-8) against the oracle; the fused path launched
    fewer kernels than the per-product path on the same run."""
    p = CASES[name]()
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=40)
    x, hist, info = tacta.cta_solve(A, b, fused_chain=1, **opts)
    _, _, info0 = tacta.cta_solve(A, b, fused_chain=0, **opts)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, **opts)
    assert info["iters"] == ref.iters == 40 and info["matvecs"] == ref.matvecs == info0["matvecs"]
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    np.testing.assert_allclose(hist.cpu().numpy(), ref.hist, rtol=1e-8)
    assert info["launches"] < info0["launches"]


@pytest.mark.parametrize("name", ["stencil_300", "rect_banded"])
def test_fused_equals_per_product_path(tacta, name):
    """The two paths differ only in the order of the moments' partial sums (relative
    differences ~1e-16), which the t x t centering solve amplifies by its condition
    number: two steps (t = 1, 2) agree to 1e-13, four (t up to 4, condition ~1e5 on the
    stencil) to 1e-10."""
    p = CASES[name]()
    A, b = dev(p)
    for steps, tol in ((2, 1e-13), (4, 1e-10)):
        opts = dict(tol=1e-30, tol_normal=0.0, max_iter=steps)
        x1, h1, _ = tacta.cta_solve(A, b, fused_chain=1, **opts)
        x0, h0, _ = tacta.cta_solve(A, b, fused_chain=0, **opts)
        x1, x0 = x1.cpu().numpy(), x0.cpu().numpy()
        assert np.linalg.norm(x1 - x0) <= tol * np.linalg.norm(x0), steps
        np.testing.assert_allclose(h1.cpu().numpy(), h0.cpu().numpy(), rtol=tol)


def test_fused_graph_replay_is_bitwise_deterministic(tacta):
    """Graph replay and direct launches of the fused chain give identical bits."""
    p = CASES["stencil_300"]()
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=100)
    xa, ha, _ = tacta.cta_solve(A, b, use_graph=1, **opts)
    xb, hb, _ = tacta.cta_solve(A, b, use_graph=1, **opts)
    xc, hc, _ = tacta.cta_solve(A, b, use_graph=0, **opts)
    assert np.array_equal(xa.cpu().numpy(), xb.cpu().numpy())
    assert np.array_equal(xa.cpu().numpy(), xc.cpu().numpy())
    assert np.array_equal(ha.cpu().numpy(), hc.cpu().numpy())


def test_fused_mixed_precision(tacta):
    """Mixed precision on the fused FP32 chain: over the first steps its history follows
    the per-product FP32 path (same FP32 products, moments summed in another order), and
    the refined solve reaches 1e-12 with x within 1e-9 of the exact solution (x* = 1)."""
    p = gen.convdiff_stencil(40)
    A, b = dev(p)
    _, h1, _ = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=8,
                               precision=tacta.PRECISION_MIXED, fused_chain=1)
    _, h0, _ = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=8,
                               precision=tacta.PRECISION_MIXED, fused_chain=0)
    np.testing.assert_allclose(h1.cpu().numpy(), h0.cpu().numpy(), rtol=1e-5)
    x, _, info = tacta.cta_solve(A, b, tol=1e-12, tol_normal=0.0, max_iter=200000,
                                 precision=tacta.PRECISION_MIXED, fused_chain=1)
    assert info["reason_name"] == "RESIDUAL" and info["rel_res"] <= 1e-12
    assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-9


def fpt_bytes(p, t, vsize=8.0):
    """Algorithmic bytes of an unfused F_t step of order t on CSR operands: t products with
    A and t with Aᵀ (values, indices, row offsets), the chain's vectors and the update."""
    ba = (vsize + 4) * p.nnz + 4 * (p.m + 1)
    bat = (vsize + 4) * p.nnz + 4 * (p.n + 1)
    return t * (ba + bat) + vsize * t * (2 * p.m + 2 * p.n) + vsize * (t + 2) * (p.n + p.m)


def test_fused_profile_counts_products(tacta):
    """profile = 1 times the fused step (fused_chain = 1, 2) as one unit per F_t step with
    the step's algorithmic bytes; the chain-only launch (fused_chain = 3) as its 2t
    products, and on the run-staged CSR the per-product path's counts and bytes."""
    p = CASES["stencil_300"]()
    A, b = dev(p)
    per_step = [1, 2, 3, 4, 5, 4, 3, 2]
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=8, profile=1)
    _, _, i1 = tacta.cta_solve(A, b, fused_chain=2, **opts)
    assert i1["spmv_count"] == 8 and i1["spmv_ms"] > 0
    assert i1["spmv_bytes"] == pytest.approx(sum(fpt_bytes(p, t) for t in per_step), rel=1e-12)
    _, _, i3 = tacta.cta_solve(A, b, fused_chain=3, **opts)
    _, _, i0 = tacta.cta_solve(A, b, fused_chain=0, **opts)
    assert i3["spmv_count"] == i0["spmv_count"] == 2 * sum(per_step)


@pytest.mark.parametrize("name", ["stencil_300", "rect_banded"])
def test_fused_step_equals_chain_with_separate_update(tacta, name):
    """The fused step (fused_chain = 1) and the chain with its auxiliary solve and update
    as separate launches (fused_chain = 3) sum the same partials in the same order and
    update every entry with the same FMAs: x is bit for bit the same; only ||r||² is
    added in another order (the history agrees to 1e-14). With R = 7 the fused step
    starts every eighth step with the true residual b - A x (its own product inside the
    launch, instead of a separate gated launch), with the same per-row arithmetic."""
    p = CASES[name]()
    A, b = dev(p)
    for R in (40, 7):
        opts = dict(tol=1e-30, tol_normal=0.0, max_iter=40, recompute_every=R)
        x1, h1, i1 = tacta.cta_solve(A, b, fused_chain=1, **opts)
        x3, h3, i3 = tacta.cta_solve(A, b, fused_chain=3, **opts)
        assert i1["iters"] == i3["iters"] == 40 and i1["launches"] < i3["launches"]
        assert i1["matvecs"] == i3["matvecs"]
        assert np.array_equal(x1.cpu().numpy(), x3.cpu().numpy()), R
        np.testing.assert_allclose(h1.cpu().numpy(), h3.cpu().numpy(), rtol=1e-14)


def test_fused_step_timeout_is_reported_and_the_plan_recovers(tacta):
    """wait_limit_log2 = 1 makes the grid-wide waits of the fused launch give up after two
    cycles: a block waiting for the others' previous product stops, the launch ends with
    the TIMEOUT reason (every armed copy drained first) and the call returns
    TACTA_ERR_TIMEOUT. The next solve on the same plan is the normal one."""
    p = CASES["stencil_300"]()
    A, b = dev(p)
    plan = tacta.Plan(A)
    try:
        opts = dict(tol=1e-30, tol_normal=0.0, max_iter=8)
        with pytest.raises(tacta.TactaError, match="TIMEOUT"):
            plan.cta(b, wait_limit_log2=1, **opts)
        x, _, info = plan.cta(b, **opts)
        ref = oracle.cta_solve(oracle.make_operator(p), p.b, **opts)
        assert info["iters"] == 8
        assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    finally:
        plan.close()



# ------------------------------------------------------------------ diagonal form

def dia_bytes(p, k, vsize=8.0):
    """Algorithmic bytes of one product on the diagonal form: k values per row of every
    256-row tile, one mask byte per row, x read once, y written once."""
    rows_t = -(-p.m // 256) * 256
    return vsize * k * rows_t + rows_t + vsize * p.n + vsize * p.m


@pytest.mark.parametrize("name", ["stencil_300", "rect_banded", "clement_5001"])
def test_diagonal_form_matches_run_staged_chain(tacta, name):
    """fused_chain = 1 runs the chain on the diagonal form (the chain-only launch of
    fused_chain = 3 profiles the diagonal form's bytes), fused_chain = 2 on the run-staged
    CSR; every row's FMAs run in the same order, so the two trajectories agree to rounding
    in the moments' partial sums (bit for bit when both launches have the same grid)."""
    p = CASES[name]()
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=8, profile=1)
    x1, h1, _ = tacta.cta_solve(A, b, fused_chain=1, **opts)
    _, _, i1 = tacta.cta_solve(A, b, fused_chain=3, **opts)
    x2, h2, i2 = tacta.cta_solve(A, b, fused_chain=2, **opts)
    S = sp.csr_matrix((p.vals, p.colidx, p.rowptr), shape=(p.m, p.n))
    rows = np.repeat(np.arange(p.m), np.diff(S.indptr))
    k = len(np.unique(S.indices - rows))
    St = S.T.tocsr()
    pt = gen.Problem(name="t", m=p.n, n=p.m, fmt="csr", rowptr=St.indptr, colidx=St.indices, vals=St.data)
    per_step = [1, 2, 3, 4, 5, 4, 3, 2]
    want = sum(t * (dia_bytes(pt, k) + dia_bytes(p, k)) for t in per_step)
    assert i1["spmv_bytes"] == pytest.approx(want, rel=1e-12)
    x1, x2 = x1.cpu().numpy(), x2.cpu().numpy()
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x2)
    np.testing.assert_allclose(h1.cpu().numpy(), h2.cpu().numpy(), rtol=1e-12)


def test_diagonal_form_mixed_precision(tacta):
    """The FP32 chain on the diagonal form: the refined solve reaches 1e-12 with x within
    1e-9 of the exact solution (x* = 1), as on the run-staged CSR."""
    p = gen.convdiff_stencil(40)
    A, b = dev(p)
    for fused in (1, 2):
        x, _, info = tacta.cta_solve(A, b, tol=1e-12, tol_normal=0.0, max_iter=200000,
                                     precision=tacta.PRECISION_MIXED, fused_chain=fused)
        assert info["reason_name"] == "RESIDUAL" and info["rel_res"] <= 1e-12
        assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-9


def test_many_diagonals_stay_on_run_staged_csr(tacta):
    """Eight diagonals (more than the diagonal form holds): fused_chain = 1 runs the
    run-staged CSR chain (its profiled bytes are the CSR's) and matches the oracle."""
    rng = np.random.default_rng(13)
    offs = [0, 1, 2, 3, 40, 41, 42, 43]
    S = sp.csr_matrix(sp.diags([rng.standard_normal(6000) for _ in offs], offs, shape=(6000, 6100)))
    S.sort_indices()
    p = from_scipy(S, 14)
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=8, profile=1)
    x, _, _ = tacta.cta_solve(A, b, fused_chain=1, **opts)
    _, _, info = tacta.cta_solve(A, b, fused_chain=3, **opts)
    _, _, info2 = tacta.cta_solve(A, b, fused_chain=0, **opts)
    assert info["spmv_bytes"] == pytest.approx(info2["spmv_bytes"], rel=1e-12)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=8)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_repeated_column_stays_on_run_staged_csr(tacta):
    """A row that stores one column twice (CSR allows it; the product adds both) cannot be
    put in diagonal form: the plan keeps the run-staged CSR chain, and the trajectory
    matches the oracle's, whose product adds the repeated entries too."""
    S = sp.csr_matrix(sp.diags([np.full(3000, 4.0), np.full(3000, -1.0), np.full(3000, -1.5)], [0, 1, -1],
                               shape=(3000, 3000)))
    S.sort_indices()
    rp, ci, va = S.indptr.copy(), list(S.indices), list(S.data)
    k = rp[5] + 1                       # row 5 stores column 5 (its diagonal) a second time
    ci.insert(k, 5)
    va.insert(k, 0.25)
    rp[6:] += 1
    rng = np.random.default_rng(3)
    p = gen.Problem(name="dup", m=3000, n=3000, fmt="csr", rowptr=rp.astype(np.int32),
                    colidx=np.array(ci, dtype=np.int32), vals=np.array(va), b=rng.standard_normal(3000))
    A, b = dev(p)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=8, profile=1)
    x, _, _ = tacta.cta_solve(A, b, fused_chain=1, **opts)
    _, _, info = tacta.cta_solve(A, b, fused_chain=3, **opts)
    _, _, info2 = tacta.cta_solve(A, b, fused_chain=0, **opts)
    assert info["spmv_bytes"] == pytest.approx(info2["spmv_bytes"], rel=1e-12)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=8)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
