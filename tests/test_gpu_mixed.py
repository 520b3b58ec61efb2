"""Mixed-precision CTA (FP32 chain, FP64 centering solve, stop tests and refinement)
against the FP64 oracle (needs a GB300).

The FP32 path follows a different rounding trajectory by design, so it is judged
on what the refinement guarantees: the true FP64 residual meets the tolerance,
and the solution matches the FP64 oracle's converged solution (and the known
exact solution) within the bound stated in each test.
"""
import numpy as np
import pytest

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


def dev(p):
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    return (t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n)),
            torch.from_numpy(np.ascontiguousarray(p.b)).to(d))


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N", [12, 40])
def test_mixed_stencil_reaches_fp64_accuracy(tacta, N):
    """Stencil with x* = 1: the refined mixed solve reaches 1e-12 true residual and the
    solution agrees with the FP64 oracle's to 1e-9 (both are within kappa * 1e-12 of 1)."""
    p = gen.convdiff_stencil(N)
    A, b = dev(p)
    x, hist, info = tacta.cta_solve(A, b, tol=1e-12, tol_normal=0.0, max_iter=200000,
                                    precision=tacta.PRECISION_MIXED)
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-12, tol_normal=0.0, max_iter=200000)
    xg = x.cpu().numpy()
    assert info["reason_name"] == "RESIDUAL" and info["rel_res"] <= 1e-12
    assert np.abs(xg - 1.0).max() <= 1e-9
    assert relerr(xg, ref.x) <= 1e-9


def test_mixed_matches_fp64_gpu_residual_history_early(tacta):
    """Over the first climb of the t-cycle the mixed residual history follows the FP64
    one: to 1e-5 for t = 1, 2 and to 1e-3 once t = 3..5 moments (FP32 vectors) enter."""
    p = gen.convdiff_stencil(64)
    A, b = dev(p)
    _, h64, _ = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=8)
    _, h32, _ = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=8,
                                precision=tacta.PRECISION_MIXED)
    h64, h32 = h64.cpu().numpy(), h32.cpu().numpy()
    np.testing.assert_allclose(h32[:3], h64[:3], rtol=1e-5)
    np.testing.assert_allclose(h32, h64, rtol=1e-3)


def test_mixed_clement_singular(tacta):
    """Singular Clement (b in range): the true residual meets 1e-10; the solution differs
    from the minimum-norm one by at most 1e-6 relative -- FP32 rounding puts components in
    the null space that no residual can see (stated error of the mixed path)."""
    p = gen.clement(1001)
    A, b = dev(p)
    x, hist, info = tacta.cta_solve(A, b, tol=1e-10, tol_normal=0.0, max_iter=400000,
                                    precision=tacta.PRECISION_MIXED)
    D = p.to_dense()
    xs = np.linalg.pinv(D, rcond=1e-10) @ p.b
    assert info["reason_name"] == "RESIDUAL" and info["rel_res"] <= 1e-10
    assert relerr(x.cpu().numpy(), xs) <= 1e-6


def test_mixed_rejects_dense(tacta):
    import torch
    q = gen.dense_gaussian(20, 20, seed=1)
    A = torch.from_numpy(q.dense).to("cuda:0")
    b = torch.from_numpy(q.b).to("cuda:0")
    with pytest.raises(tacta.TactaError, match="CSR"):
        tacta.cta_solve(A, b, precision=tacta.PRECISION_MIXED)


def test_mixed_large_norm_matrix_stays_finite(tacta):
    """The FP32 chain is scaled by a power of two near 1/||A||: the Clement matrix of
    order 20001 (||A|| = 2e4, so (AAᵀ)^5 r would overflow FP32) runs without overflow and
    its residual decreases like the FP64 path's over a fixed budget."""
    p = gen.clement(20001)
    A, b = dev(p)
    _, h32, i32 = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=400,
                                  precision=tacta.PRECISION_MIXED)
    _, h64, i64 = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=400)
    assert i32["status"] == 1 and np.isfinite(i32["rel_res"])
    assert i32["rel_res"] <= 3.0 * i64["rel_res"]
