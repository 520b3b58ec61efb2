"""bench.py's host arithmetic, on the CPU: the algorithmic bytes its roofline divides by
(the survey's per-product and per-F_t-step formulas, checked against their worked value
for the 1000² stencil), the step-order schedule it uses for the mean t (against the
oracle's Sec. 5.1 schedule), and the batched completion profile (closed forms)."""
import numpy as np
import pytest

import bench
import oracle


def test_bytes_per_product_and_per_fpt_on_the_stencil():
    n = m = 1000 * 1000
    nnz = 5 * n - 4 * 1000          # the 5-point stencil on a 1000 x 1000 grid
    assert nnz == 4_996_000
    # 12 nnz (values, column indices) + 4 (m + 1) (row offsets) + 8 n (x) + 8 m (y)
    assert bench.survey_bytes_per_product(m, n, nnz) == 79_952_004
    # t (B_A + B_At) + 8 t (m + 2n + m) + 8 (t + 2)(n + m) at t = 3: ~560 MB per F_t step
    assert bench.survey_bytes_per_fpt(m, n, nnz, 3) == 559_712_024
    # t = 1: one product with each of A and Aᵀ, the chain's vectors once, the update
    assert bench.survey_bytes_per_fpt(m, n, nnz, 1) == 2 * 63_952_004 + 8 * 4e6 + 24 * 2e6


def test_fpt_schedule_is_the_oracles_ping_pong():
    for t_max in (2, 3, 5, 8):
        want = [oracle.schedule(k, t_max) for k in range(40)]
        assert [bench.fpt_schedule(k, t_max) for k in range(40)] == want, t_max
    assert [bench.fpt_schedule(k) for k in range(9)] == [1, 2, 3, 4, 5, 4, 3, 2, 1]


def test_completion_profile_closed_forms():
    ms = 1_000_000   # ns
    tb = np.array([0, 0, 10, 10]) * ms
    te = np.array([10, 10, 20, 30]) * ms
    p = bench.completion_profile(tb, te, blocks=2)
    assert (p["p50_ms"], p["p90_ms"], p["p99_ms"], p["p100_ms"]) == (10.0, 30.0, 30.0, 30.0)
    assert p["longest_system_ms"] == 20.0
    assert p["busy_frac"] == pytest.approx(50.0 / 60.0)      # 50 ms of systems in 2 x 30 ms
    assert p["tail_busy_frac"] is None                       # nothing after the 90 % mark
    q = bench.completion_profile(tb, te, blocks=2, clustered=True)
    assert "busy_frac" not in q and q["p100_ms"] == 30.0
