"""Enhanced CTA (Sec. 3.2, Eq. widehatxB) on the GPU against the oracle (needs a GB300).

The device evaluates the first-order iterates' quadratic forms from the step's moments;
the oracle forms the iterates as vectors. Early stops are compared step for step; late
ones (hundreds of steps, beyond what two summation orders reproduce) by what the stop
guarantees: reason, the normal-equation residual at the tolerance, and the residual
matching b - A x.
"""
import numpy as np
import pytest

import gen
import oracle
import oracle.cta as ocx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tacta():
    import torch
    import paper_2304_12168_gb300 as t
    t.load_library()
    torch.cuda.set_device(0)
    return t


def system(seed, m=60, n=90):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, 8)) @ rng.standard_normal((8, n)) + 0.05 * rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n)
    return gen.Problem(name="e", m=m, n=n, fmt="dense", dense=np.ascontiguousarray(A), b=b)


def solve(tacta, p, **opts):
    import torch
    A = torch.from_numpy(p.dense).to("cuda:0")
    b = torch.from_numpy(p.b).to("cuda:0")
    x, hist, info = tacta.cta_solve(A, b, **opts)
    return x.cpu().numpy(), hist.cpu().numpy(), info


def test_enhanced_closed_form(tacta):
    """A = 2Q, Q orthogonal 64 x 64: the first first-order iterate vanishes, so the
    enhanced algorithm stops after one step with x = A^{-1} b. Its test value
    r_1ᵀ H r_1 = phi_1 - 2 a phi_2 + a² phi_3 cancels to rounding (~1e-16 phi_1), which the
    test resolves for tol_normal down to ~1e-7 (the reading of Sec. 3.2's test): 1e-6."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((64, 64)))
    b = rng.standard_normal(64)
    p = gen.Problem(name="q", m=64, n=64, fmt="dense", dense=np.ascontiguousarray(2.0 * Q), b=b)
    x, _, info = solve(tacta, p, tol=1e-30, tol_normal=1e-6, max_iter=5, t_max=2, cycle=2, enhanced=1)
    assert info["reason_name"] == "ENHANCED" and info["iters"] == 1
    np.testing.assert_allclose(x, Q.T @ b / 2.0, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2])
def test_enhanced_early_stop_matches_oracle(tacta, seed):
    """tol_normal = 1e-3: the enhanced stop fires within the first steps; same step, reason,
    history and x as the oracle."""
    p = system(seed)
    opts = dict(tol=1e-30, tol_normal=1e-3, max_iter=500)
    x, hist, info = solve(tacta, p, enhanced=1, **opts)
    ref = ocx.cta_solve(oracle.make_operator(p), p.b, enhanced=True, **opts)
    assert ref.reason == oracle.Reason.ENHANCED
    assert info["reason_name"] == "ENHANCED" and info["iters"] == ref.iters
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    np.testing.assert_allclose(hist, ref.hist, rtol=1e-8)


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_enhanced_late_stop_properties(tacta, seed):
    """tol_normal = 1e-5 (hundreds of steps): the GPU stops by the enhanced test or the
    plain normal-equation test, with the true normal-equation residual at the tolerance,
    and no later than the plain algorithm's stop."""
    p = system(seed)
    opts = dict(tol=1e-30, tol_normal=1e-5, max_iter=2000)
    x, _, info = solve(tacta, p, enhanced=1, **opts)
    _, _, plain = solve(tacta, p, enhanced=0, **opts)
    assert info["reason_name"] in ("ENHANCED", "NORMAL")
    A = p.dense
    nr = np.linalg.norm(A.T @ (p.b - A @ x)) / np.linalg.norm(A.T @ p.b)
    assert nr <= 1e-5 * (1 + 1e-3)
    assert info["iters"] <= plain["iters"]
