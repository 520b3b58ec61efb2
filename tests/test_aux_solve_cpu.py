"""The auxiliary solve the kernels run (Eq. eqcoeff), built for the host and called through
tacta_aux_solve, against the oracle and what the mathematics fixes (no GPU needed)."""
import numpy as np
import pytest

import oracle.cta as ocx
import paper_2304_12168_gb300 as tacta


@pytest.fixture(scope="module")
def lib():
    try:
        return tacta.load_library()
    except RuntimeError as e:
        pytest.skip(str(e))


def moments(A, r, t):
    """phi_{2i-1} = ||z_i||², phi_{2i} = ||u_i||² of the chain u_0 = r, z_i = Aᵀu_{i-1}, u_i = A z_i."""
    phi = np.zeros(2 * t + 1)
    u = r
    for i in range(1, t + 1):
        z = A.T @ u
        u = A @ z
        phi[2 * i - 1] = z @ z
        phi[2 * i] = u @ u
    return phi


def cases(seed, count):
    rng = np.random.default_rng(seed)
    for trial in range(count):
        n = int(rng.integers(2, 30))
        t = int(rng.integers(1, 9))
        if trial % 3 == 0:
            A = rng.standard_normal((n, n))
        elif trial % 3 == 1:          # low rank: the Hankel matrix turns singular at order rank + 1
            k = max(1, n // 4)
            A = rng.standard_normal((n, k)) @ rng.standard_normal((k, n))
        else:                         # few distinct singular values: exact truncation
            A = np.diag(rng.choice([0.5, 1.0, 2.0], n))
        r = rng.standard_normal(n) * 10.0 ** rng.uniform(-30, 30)
        yield t, moments(A, r, t)


def test_matches_oracle_rank_and_solves_its_leading_block(lib):
    """Same truncation order as the oracle; the leading block's backward error (Jacobi-scaled)
    is at rounding level whatever its conditioning; well-conditioned orders agree with the
    oracle's alpha to 1e-9."""
    for t, phi in cases(0, 1500):
        a_o, r_o = ocx.hankel_solve(phi, t, 1e-12)
        a_c, r_c = tacta.aux_solve(phi, t, 1e-12)
        assert r_c == r_o, (t, r_o, r_c)
        assert np.all(a_c[r_c:] == 0.0)
        if r_c == 0:
            continue
        H = np.array([[phi[i + j + 2] for j in range(r_c)] for i in range(r_c)])
        rhs = phi[1:r_c + 1]
        d = 1.0 / np.sqrt(np.diag(H))
        res = d * (H @ a_c[:r_c] - rhs)
        scale = np.abs(d[:, None] * H * d[None, :]) @ np.abs(a_c[:r_c] / d) + np.abs(d * rhs)
        assert np.all(np.abs(res) <= 1e-12 * scale.max()), (t, r_c)
        if r_c <= 2:
            np.testing.assert_allclose(a_c, np.asarray(a_o), rtol=1e-9, atol=0)


def test_order_one_closed_form(lib):
    """t = 1: alpha = phi_1 / phi_2 (Eq. eqcoeff with one unknown)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        phi = np.array([0.0, *(10.0 ** rng.uniform(-100, 100, 2))])
        a, r = tacta.aux_solve(phi, 1)
        assert r == 1 and a[0] == pytest.approx(phi[1] / phi[2], rel=4e-16)


def test_breakdown_and_bad_arguments(lib):
    a, r = tacta.aux_solve(np.zeros(11), 5)
    assert r == 0 and np.all(a == 0.0)
    with pytest.raises(ValueError):
        tacta.aux_solve(np.zeros(19), 9)
