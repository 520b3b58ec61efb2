"""The batched solve's schedule model (tacta_batch_simulate_makespan), on the host: the
planner predicts a solve's makespan with it when it decides which systems thread-block
clusters take. Checked against closed forms and against plain list scheduling written
out here with a heap."""
import heapq
import os

import numpy as np
import pytest

import paper_2304_12168_gb300 as tacta
from paper_2304_12168_gb300 import build as tbuild


@pytest.fixture(scope="module")
def sim():
    if not os.path.exists(tacta.LIB_PATH):
        tbuild.build()
    tacta.load_library()
    return tacta.Batch.simulate_makespan


def list_schedule(w, clusters, C, d, sms, per_sm):
    """Longest first onto the earliest free cluster; then blocks: per_sm on every free SM
    at 0, per_sm on each of a cluster's C SMs when it finishes; longest first onto the
    earliest free block."""
    end = 0.0
    cq = [0.0] * clusters
    for v in sorted(w, reverse=True):
        t = heapq.heappop(cq)
        heapq.heappush(cq, t + v)
        end = max(end, t + v)
    bq = [0.0] * ((sms - clusters * C) * per_sm) + [t for t in cq for _ in range(C * per_sm)]
    heapq.heapify(bq)
    for v in sorted(d, reverse=True):
        t = heapq.heappop(bq)
        heapq.heappush(bq, t + v)
        end = max(end, t + v)
    return end


def test_closed_forms(sim):
    # k rounds of equal jobs on every block
    assert sim([], 0, 1, [1.0] * (3 * 152 * 2), 152, 2) == 3.0
    # one job longer than all the others together spread over the blocks
    assert sim([], 0, 1, [500.0] + [1.0] * 1000, 152, 1) == 500.0
    # a cluster job alone
    assert sim([10.0], 1, 8, [], 152, 1) == 10.0
    # every SM in the cluster: the blocks start when it finishes (16 unit jobs, 8 blocks)
    assert sim([10.0], 1, 8, [1.0] * 16, 8, 1) == 12.0
    # two clusters of 4 on 8 SMs, jobs 6 and 2: the blocks of the second start at 2
    # (4 blocks take four jobs of 4: ends at 6)
    assert sim([6.0, 2.0], 2, 4, [4.0] * 4, 8, 1) == 6.0
    # past the 512 longest one-block jobs the rest is spread as a fluid (equal jobs: exact)
    assert sim([], 0, 1, [1.0] * 1000, 4, 1) == 250.0


def test_against_list_scheduling(sim):
    rng = np.random.default_rng(0)
    for _ in range(200):
        sms = int(rng.integers(1, 40))
        per_sm = int(rng.integers(1, 4))
        C = int(rng.choice([1, 2, 4, 8]))
        clusters = int(rng.integers(0, sms // C + 1))
        w = list(rng.exponential(5.0, int(rng.integers(0, 6)))) if clusters else []
        d = list(rng.exponential(1.0, int(rng.integers(0, 300))))
        got = sim(w, clusters, C, d, sms, per_sm)
        want = list_schedule(w, clusters, C, d, sms, per_sm)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12), (sms, per_sm, C, clusters, len(w), len(d))


def test_fluid_tail_bounds(sim):
    """Beyond 512 one-block jobs the model is water filling: never below the lower bounds
    (the longest job; the total work over the blocks) and never above the list schedule's
    end plus the longest fluid job."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        sms, per_sm = 152, int(rng.integers(1, 3))
        d = list(np.concatenate([rng.exponential(20.0, 100), rng.exponential(1.0, 3000)]))
        got = sim([], 0, 1, d, sms, per_sm)
        assert got >= max(d) - 1e-9 and got >= sum(d) / (sms * per_sm) - 1e-9
        tail = sorted(d, reverse=True)[512:]
        assert got <= list_schedule([], 0, 1, d, sms, per_sm) + max(tail) + 1e-9


def test_invalid_arguments(sim):
    assert sim([1.0], 0, 1, [], 8, 1) == -1.0          # cluster jobs without clusters
    assert sim([], 3, 4, [], 8, 1) == -1.0             # 12 SMs of clusters on 8
    assert sim([], 0, 1, [-1.0], 8, 1) == -1.0         # negative time
    assert sim([], 0, 1, [float("nan")], 8, 1) == -1.0
    assert sim([], 0, 0, [], 8, 1) == -1.0             # cluster size 0
    assert sim([], 0, 1, [], 0, 1) == -1.0             # no SMs


# ------------------------------------------------------------ the planner's choices

SIZES = (16, 8, 4, 2, 1)
ALL_FIT = dict(max_clusters=[7, 15, 30, 60, 152], a_cap=[10**7] * 5)   # every size fits, rows staged


def plan(dur, steps, m, n, storage=1, **kw):
    args = dict(ALL_FIT, t_max=5, cycle=0, sms=152, per_sm=1)
    args.update(kw)
    return tacta.Batch.plan_search(dur, steps, m, n, storage, **args)


def long_tail_batch(n_long=4, m_long=400, long_ms=2000.0):
    """1000 one-millisecond systems and n_long systems of long_ms that take 20000 steps."""
    dur = np.array([1e6] * 1000 + [long_ms * 1e6] * n_long)
    steps = np.array([100] * 1000 + [20000] * n_long)
    m = np.array([64] * 1000 + [m_long] * n_long)
    return dur, steps, m, m.copy()


def test_planner_without_times_or_clusters(sim):
    dur, steps, m, n = long_tail_batch()
    ms, p, order = plan(np.zeros_like(dur), steps, m, n)
    assert (ms, p) == (0.0, (0, 0, 0)) and np.array_equal(order, np.arange(len(dur)))
    ms, p, order = plan(dur, steps, m, n, wide_mode=0)
    assert p == (0, 0, 0) and ms == pytest.approx(2000.0)          # the longest system on one block
    assert set(order[:4]) == {1000, 1001, 1002, 1003}               # longest first
    assert ms == pytest.approx(sim([], 0, 1, dur, 152, 1) * 1e-6)


def test_planner_puts_the_long_tail_on_clusters(sim):
    """Four systems of 2 s (20000 steps) among 1000 of 1 ms: clusters take exactly the four,
    they head the queue, and the predicted makespan lies between its lower bound (the
    largest of one-block time / 16 and the balanced time) and the one-block makespan."""
    dur, steps, m, n = long_tail_batch()
    ms, (k, c, cl), order = plan(dur, steps, m, n)
    assert k == 4 and c in SIZES[:4] and 1 <= cl <= 4
    assert set(order[:4]) == {1000, 1001, 1002, 1003}
    assert sorted(order) == list(range(len(dur)))
    assert max(2000.0 / 16, dur.sum() * 1e-6 / 152) < ms < 0.98 * 2000.0


def test_planner_respects_row_count_and_fit():
    """A cluster of C blocks needs at least 4C rows: 40-row systems can go to clusters of 8
    at most. A size whose vectors do not fit (max_clusters 0) is never chosen."""
    dur, steps, m, n = long_tail_batch(m_long=40)
    ms, (k, c, cl), _ = plan(dur, steps, m, n)
    assert k == 4 and c <= 8
    ms2, (k2, c2, _), _ = plan(dur, steps, m, n, max_clusters=[7, 0, 30, 60, 152])
    assert k2 == 4 and c2 in (4, 2)


def test_planner_prices_streamed_rows():
    """Rows that do not fit a block's shared memory are streamed: with no staging room the
    predicted makespan does not improve, and for FP64 rows it grows."""
    dur, steps, m, n = long_tail_batch(m_long=512)
    ms_staged, p_staged, _ = plan(dur, steps, m, n, storage=0)
    ms_stream, p_stream, _ = plan(dur, steps, m, n, storage=0, a_cap=[0] * 5)
    assert p_staged[0] == 4 and ms_stream >= ms_staged


def test_planner_leaves_balanced_batches_alone():
    dur = np.full(2000, 5e6)
    ms, p, _ = plan(dur, np.full(2000, 500), np.full(2000, 300), np.full(2000, 300))
    assert p == (0, 0, 0) and ms > 0


def test_planner_forced_plans():
    dur, steps, m, n = long_tail_batch()
    ms, p, order = plan(dur, steps, m, n, wide_mode=3, wide_cluster=4)
    assert p == (3, 4, 3) and set(order[:3]) <= {1000, 1001, 1002, 1003}
    ms, p, _ = plan(dur, steps, m, n, wide_mode=3, wide_cluster=4, wide_clusters=2)
    assert p == (3, 4, 2)
    ms, p, _ = plan(dur, steps, m, n, wide_mode=3)           # the largest size that fits
    assert p == (3, 16, 3)
    ms, p, _ = plan(dur, steps, m, n, wide_mode=3, wide_cluster=16, max_clusters=[0, 15, 30, 60, 152])
    assert p == (0, 0, 0) and ms == float("inf")
    ms, p, _ = plan(np.zeros_like(dur), steps, m, n, wide_mode=2, wide_cluster=8)   # before any times
    assert p == (2, 8, 2) and ms == 0.0


def test_planner_invalid_arguments():
    dur, steps, m, n = long_tail_batch()
    assert plan(dur, steps, m, n, storage=7)[0] == -1.0
    assert plan(dur, steps, m, n, t_max=0)[0] == -1.0
    assert plan(dur, steps, m, n, wide_mode=-2)[0] == -1.0
    assert plan(dur, steps, m, n, wide_cluster=32)[0] == -1.0
    assert plan(dur, steps, m, n, h0=float("nan"))[0] == -1.0
    bad = dur.copy(); bad[0] = -1.0
    assert plan(bad, steps, m, n)[0] == -1.0
    bad_m = m.copy(); bad_m[3] = 0
    assert plan(dur, steps, bad_m, n)[0] == -1.0
