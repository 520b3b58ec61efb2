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


def _device(p):
    import torch
    import paper_2304_12168_gb300 as t
    d = torch.device("cuda:0")
    b = torch.from_numpy(np.ascontiguousarray(p.b)).to(d)
    if p.fmt == "dense":
        return torch.from_numpy(np.ascontiguousarray(p.dense)).to(d), b
    return t.CSR(torch.from_numpy(p.rowptr).to(d), torch.from_numpy(p.colidx).to(d),
                 torch.from_numpy(p.vals).to(d), (p.m, p.n)), b


@pytest.mark.parametrize("kind", ["csr", "dense"])
def test_residual_static_matches_cta_solve_on_two_calls_in_a_row(kind):
    import torch
    import paper_2304_12168_gb300 as tacta
    tacta.load_library()
    torch.cuda.set_device(0)
    p = gen.convdiff_stencil(60) if kind == "csr" else gen.dense_gaussian(300, 200, seed=4)
    A, b = _device(p)
    bnorm = float(torch.linalg.norm(b))
    rng = np.random.default_rng(3)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal(p.n)).to("cuda:0")
        # the existing entry point: cta_solve from x0 = x with no iterations reports the
        # true residual b - A x at exit
        _, hist, info = tacta.cta_solve(A, b, x, tol=1e-30, tol_normal=0.0, max_iter=0)
        r, rr, rb = tacta.residual_static(A, x, b)
        assert abs(np.sqrt(rr) / bnorm - info["rel_res"]) <= RES_TOL * max(1.0, info["rel_res"])
        assert abs(np.sqrt(rr) / bnorm - float(hist[0])) <= RES_TOL * max(1.0, float(hist[0]))
        # r itself is b - A x, and rᵀb is its dot with b
        assert float(torch.linalg.norm(r)) ** 2 == pytest.approx(rr, rel=1e-12)
        assert float(torch.dot(r, b)) == pytest.approx(rb, rel=1e-10, abs=1e-10 * bnorm ** 2)


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
