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
