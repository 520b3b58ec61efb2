"""tacta_residual_static: the allocation-free residual entry point, through the C ABI.

Some callers cannot allocate device memory at the point of the call (a framework
whose caching allocator owns the device; latency-bound loops that must not enter
cudaMalloc). For them the library offers tacta_residual_static, whose reduction
scratch is a file-scope device array instead of plan workspace. This file is
collected last so that, should it fail, a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu

RES_TOL = 1e-10      # final relative residuals agree within 1e-10 (as in test_gpu_parity)
U = np.finfo(np.float64).eps / 2


def _device(p):
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    b = torch.from_numpy(np.ascontiguousarray(p.b)).to(d)
    if p.fmt == "dense":
        return torch.from_numpy(np.ascontiguousarray(p.dense)).to(d), b
    return t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                 torch.from_numpy(p.vals).to(d), (p.m, p.n)), b


def _host_residual(p, x):
    """b - A x on the host in FP64, and the rounding bound of one side per row:
    (k + 1) u (|b| + |A||x|) with k the row's stored entries."""
    S = p.scipy()
    r = p.b - S @ x
    absS = abs(S)
    k = np.diff(S.indptr) if p.fmt == "csr" else np.full(p.m, p.n)
    bound = (k + 1) * U * (np.abs(p.b) + absS @ np.abs(x))
    return r, bound


@pytest.mark.parametrize("kind", ["csr", "dense"])
def test_residual_static_matches_cta_solve_on_two_calls_in_a_row(kind):
    import torch
    import paper_2304_12168_gb300 as tacta
    tacta.load_library()
    torch.cuda.set_device(0)
    p = gen.convdiff_stencil(60) if kind == "csr" else gen.dense_gaussian(300, 200, seed=4)
    A, b = _device(p)
    bnorm = float(np.linalg.norm(p.b))
    rng = np.random.default_rng(3)
    for call in range(2):
        xh = rng.standard_normal(p.n)
        x = torch.from_numpy(xh).to("cuda:0")
        # the existing entry point: cta_solve from x0 = x with no iterations reports the
        # true residual b - A x at exit
        _, hist, info = tacta.cta_solve(A, b, x, tol=1e-30, tol_normal=0.0, max_iter=0)
        r, rr, rb = tacta.residual_static(A, x, b)
        assert abs(np.sqrt(rr) / bnorm - info["rel_res"]) <= RES_TOL * max(1.0, info["rel_res"])
        assert abs(np.sqrt(rr) / bnorm - float(hist[0])) <= RES_TOL * max(1.0, float(hist[0]))
        # r entry by entry against b - A x formed on the host: the two sides differ by at
        # most the sum of their rounding bounds
        rh, bound = _host_residual(p, xh)
        rg = r.cpu().numpy()
        assert np.all(np.abs(rg - rh) <= 2 * bound), float(np.max(np.abs(rg - rh) / (2 * bound)))
        # the reductions against host sums of the host residual (error of a sum of m terms
        # plus the propagated per-entry bound)
        m = p.m
        assert abs(rr - float(rh @ rh)) <= 2 * float(np.abs(rh) @ (2 * bound)) + 2 * m * U * float(rh @ rh)
        assert abs(rb - float(rh @ p.b)) <= float(np.abs(p.b) @ (2 * bound)) + 2 * m * U * float(np.abs(rh) @ np.abs(p.b))


def test_residual_static_rejects_host_arrays_and_oversized_m():
    import paper_2304_12168_gb300 as tacta
    import ctypes
    lib = tacta.load_library()
    M = tacta.tacta_matrix(5, 5, 25, 0, 0, 1, None, None)     # on_device = 0
    out = (ctypes.c_double * 2)()
    st = lib.tacta_residual_static(ctypes.byref(M), 1, 1, 1, ctypes.cast(out, ctypes.c_void_p), None)
    assert st == -1 and b"on_device" in lib.tacta_last_error()
    M = tacta.tacta_matrix(16_773_121, 5, 0, 1, 1, 1, 1, 1)   # one row beyond the limit
    st = lib.tacta_residual_static(ctypes.byref(M), 1, 1, 1, ctypes.cast(out, ctypes.c_void_p), None)
    assert st == -1 and b"static-scratch limit" in lib.tacta_last_error()
