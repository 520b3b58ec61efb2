"""The on-device iteration loop (a CUDA graph WHILE node over the iteration body, needs a
GB300): with graphs the solve is one graph launch that stops when the control block
reports a stop, so no launches are enqueued past the stop; the iterates equal those of
direct launches bit for bit, and max_iter bounds the loop.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def csr(p):
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    return (t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                  torch.from_numpy(p.vals).to(d), (p.m, p.n)),
            torch.from_numpy(np.ascontiguousarray(p.b)).to(d))


@pytest.mark.parametrize("fused_chain", [0, 1])
@pytest.mark.parametrize("alg", ["cta", "ta"])
def test_graph_loop_equals_direct_launches(tacta, fused_chain, alg):
    """A solve that stops after a few dozen steps: graph (on-device loop) and direct
    launches (host polling) give the same iterations and the same x bit for bit. With one
    launch per product the polled run enqueues up to two polling chunks past the stop and
    the graph run none; the graph adds only its one-thread loop kernel per body."""
    p = gen.convdiff_stencil(48)
    A, b = csr(p)
    plan = tacta.Plan(A)
    kw = dict(tol=1e-6, tol_normal=0.0, max_iter=100000, fused_chain=fused_chain)
    fn = getattr(plan, alg)
    xg, _, ig = fn(b, use_graph=1, **kw)
    xd, _, idr = fn(b, use_graph=0, **kw)
    plan.close()
    assert ig["reason_name"] == idr["reason_name"] == "RESIDUAL"
    assert ig["iters"] == idr["iters"]
    assert np.array_equal(xg.cpu().numpy(), xd.cpu().numpy())
    # the graph adds one loop kernel per body (64 steps, or one fused launch) and never
    # enqueues work past the stop; the polled run may overshoot by up to two chunks
    bodies = ig["iters"] // 64 + 2 if fused_chain == 0 or alg == "ta" else idr["launches"]
    assert ig["launches"] <= idr["launches"] + bodies


@pytest.mark.parametrize("max_iter", [0, 1, 5, 70, 130])
def test_graph_loop_stops_at_max_iter(tacta, max_iter):
    """tol = 1e-30 never passes: the loop ends after exactly max_iter steps (the device's
    MAXITER stop), across body boundaries (bodies of 64 steps)."""
    p = gen.convdiff_stencil(24)
    A, b = csr(p)
    x, _, info = tacta.cta_solve(A, b, tol=1e-30, tol_normal=0.0, max_iter=max_iter, use_graph=1)
    assert info["iters"] == max_iter and info["reason_name"] == "MAXITER"


def test_dense_graph_loop(tacta):
    """Dense A (one launch per product, FP64 and mixed): the solve stops at the same step
    with and without graphs, with the same x (bit for bit in FP64)."""
    import torch
    p = gen.dense_gaussian(120, 200, seed=4)
    A = torch.from_numpy(p.dense).to("cuda:0")
    b = torch.from_numpy(p.b).to("cuda:0")
    for prec in (tacta.PRECISION_FP64, tacta.PRECISION_MIXED):
        kw = dict(tol=1e-10, tol_normal=0.0, max_iter=5000, precision=prec, fused_chain=0)
        xg, _, ig = tacta.cta_solve(A, b, use_graph=1, **kw)
        xd, _, idr = tacta.cta_solve(A, b, use_graph=0, **kw)
        assert ig["iters"] == idr["iters"] and ig["reason_name"] == "RESIDUAL"
        assert np.array_equal(xg.cpu().numpy(), xd.cpu().numpy())
