"""Batched dense CTA (one persistent launch over many systems) against the oracle and
the mathematics (needs a GB300).

FP64 storage follows the FP64 iteration, so fixed-length trajectories must match the
oracle's per system. FP32 and BF16 storage are checked through what holds at any
precision: the FP64 residual recomputed on the host reaches the tolerance, and the
solution is the minimum-norm one (numpy pseudo-inverse) up to the storage's roundoff
times the system's condition number.
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


def small_batch(seed, count, m_range=(20, 120), aspect=None):
    """Seeded systems; aspect=(lo, hi) restricts n/m away from 1 (well conditioned)."""
    rng = np.random.default_rng(seed)
    mats, bs, lr = [], [], []
    for s in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        if aspect is None:
            n = int(rng.integers((m + 1) // 2, 2 * m + 1))
        else:
            f = rng.uniform(*aspect) if rng.random() < 0.5 else 1.0 / rng.uniform(*aspect)
            n = max(1, int(round(m * f)))
        low = s % 5 == 3
        if low:
            r = max(1, m // 2)
            A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n)) / np.sqrt(r)
        else:
            A = rng.standard_normal((m, n))
        mats.append(A)
        bs.append(A @ rng.standard_normal(n))
        lr.append(low)
    return mats, bs, np.array(lr)


def problem(A, b):
    return gen.Problem(name="d", m=A.shape[0], n=A.shape[1], fmt="dense",
                       dense=np.ascontiguousarray(A), b=b)


STREAMED = 5   # launch configuration of the fused-pass kernel with the bulk-copy ring
TENSOR = 6     # the same kernel with the products on the tensor cores (BF16 storage)


def run(tacta, mats, bs, storage, config=None, **opts):
    B = tacta.Batch(mats, storage=storage)
    if config is not None:
        B.set_config(config)
    x, iters, rel, reason = B.cta(np.concatenate(bs), **opts)
    xs = B.split(x)
    B.close()
    return xs, iters, rel, reason


@pytest.mark.parametrize("config", [None, STREAMED])
def test_fp64_fixed_trajectories_match_oracle(tacta, config):
    """Four steps (t = 1..4) per system, FP64 storage: x, iteration and product counts of
    every system against the oracle's run on that system alone; the default kernel and
    the fused-pass kernel (whose largest systems here stream through the ring)."""
    mats, bs, _ = small_batch(1, 40)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=4)
    xs, iters, rel, reason = run(tacta, mats, bs, tacta.BATCH_FP64, config=config, **opts)
    for s, (A, b) in enumerate(zip(mats, bs)):
        ref = oracle.cta_solve(oracle.make_operator(problem(A, b)), b, **opts)
        assert iters[s] == ref.iters, s
        assert np.linalg.norm(xs[s] - ref.x) <= 1e-9 * np.linalg.norm(ref.x), s
        assert rel[s] == pytest.approx(ref.rel_res, rel=1e-9), s
        assert tacta.REASON[int(reason[s])] == "MAXITER"


@pytest.mark.parametrize("config", [None, STREAMED, TENSOR])
@pytest.mark.parametrize("storage,tol,xtol", [("BATCH_FP64", 1e-10, 1e-8), ("BATCH_FP32", 1e-8, 1e-6),
                                              ("BATCH_BF16", 1e-8, 3e-2)])
def test_to_tolerance_min_norm(tacta, storage, tol, xtol, config):
    """Well-conditioned systems (n/m in [1.4, 2] or its inverse; every fifth of rank m/2):
    the host-recomputed FP64 residual meets tol, the reported one equals it, and x is the
    minimum-norm solution within cond(A) times xtol: about 100 tol for FP64, and for the
    low-precision copies 10 times their unit roundoff (2^-24, 2^-9) plus the tolerance."""
    if config == TENSOR and storage != "BATCH_BF16":
        pytest.skip("the tensor-core passes read BF16 storage only")
    mats, bs, lr = small_batch(2, 48, aspect=(1.4, 2.0))
    if config in (STREAMED, TENSOR):   # add systems larger than the shared-memory area: they stream
        m2, b2, _ = small_batch(6, 12, m_range=(220, 300), aspect=(1.4, 1.8))
        mats, bs = mats + m2, bs + b2
    xs, iters, rel, reason = run(tacta, mats, bs, getattr(tacta, storage), config=config, tol=tol,
                                 tol_normal=0.0, max_iter=20000)
    for s, (A, b) in enumerate(zip(mats, bs)):
        assert tacta.REASON[int(reason[s])] == "RESIDUAL", (s, reason[s], rel[s])
        r = np.linalg.norm(b - A @ xs[s]) / np.linalg.norm(b)
        assert r <= tol * (1 + 1e-6), (s, r)
        assert rel[s] == pytest.approx(r, rel=1e-6, abs=1e-14)
        sv = np.linalg.svd(A, compute_uv=False)
        sv = sv[sv > 1e-10 * sv[0]]
        kappa = sv[0] / sv[-1]
        xmn = np.linalg.pinv(A, rcond=1e-10) @ b
        err = np.linalg.norm(xs[s] - xmn) / np.linalg.norm(xmn)
        assert err <= xtol * kappa, (s, kappa, err)


def test_edge_cases(tacta):
    """1 x 1, one row, one column, a zero right-hand side, and max_iter = 0."""
    rng = np.random.default_rng(3)
    mats = [np.array([[2.0]]), rng.standard_normal((1, 7)), rng.standard_normal((9, 1)),
            rng.standard_normal((30, 40))]
    bs = [np.array([4.0]), rng.standard_normal(1), mats[2] @ np.array([1.5]), np.zeros(30)]
    xs, iters, rel, reason = run(tacta, mats, bs, tacta.BATCH_FP64, tol=1e-12, tol_normal=0.0, max_iter=1000)
    assert xs[0][0] == pytest.approx(2.0, rel=1e-14)
    xmn = np.linalg.pinv(mats[1]) @ bs[1]
    np.testing.assert_allclose(xs[1], xmn, rtol=1e-10, atol=1e-12)
    assert xs[2][0] == pytest.approx(1.5, rel=1e-10)
    assert tacta.REASON[int(reason[3])] == "ZERO_RHS" and np.all(xs[3] == 0.0) and iters[3] == 0
    xs, iters, rel, reason = run(tacta, mats[:3], bs[:3], tacta.BATCH_FP32, tol=1e-8, tol_normal=0.0, max_iter=0)
    assert all(tacta.REASON[int(r)] == "MAXITER" for r in reason)
    assert np.all(iters == 0) and np.allclose(rel, 1.0) and all(np.all(x == 0.0) for x in xs)


def test_empty_batch(tacta):
    B = tacta.Batch([], storage=tacta.BATCH_FP32)
    x, iters, rel, reason = B.cta(np.zeros(0))
    assert x.size == 0 and iters.size == 0
    B.close()


def test_graph_replay_and_configs_agree(tacta):
    """Graph replay and direct launch give identical results; every launch configuration
    (different block sizes, hence reduction orders) meets the tolerance; the autotuner
    picks one of them."""
    mats, bs, _ = small_batch(4, 30, m_range=(32, 200), aspect=(1.4, 2.0))
    b = np.concatenate(bs)
    B = tacta.Batch(mats, storage=tacta.BATCH_FP32)
    B.set_wide(0)   # the planner would move the longest systems onto clusters (other sums)
    opts = dict(tol=1e-8, tol_normal=0.0, max_iter=5000)
    x1, it1, r1, _ = B.cta(b, use_graph=1, **opts)
    x2, it2, r2, _ = B.cta(b, use_graph=1, **opts)
    x3, it3, r3, _ = B.cta(b, use_graph=0, **opts)
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3) and np.array_equal(it1, it3)
    tc = tacta.Batch.tensor_core_configs()
    assert TENSOR in tc
    for c in range(len(tacta.Batch.configs())):
        B.set_config(c)
        if c in tc:   # BF16 storage only: refused for this FP32 batch
            with pytest.raises(tacta.TactaError):
                B.cta(b, **opts)
            continue
        _, _, rc, reason = B.cta(b, **opts)
        assert all(tacta.REASON[int(r)] == "RESIDUAL" for r in reason) and np.all(rc <= 1e-8 * (1 + 1e-6))
    best, ms = B.tune(b, **opts)
    assert 0 <= best < len(tacta.Batch.configs()) and best not in tc and ms > 0
    B.close()


def bf16_round(a):
    """Round-to-nearest-even to BF16 (8 significant bits) of float64 values, as float64."""
    m, e = np.frexp(a)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


# shapes that reach every work split of the tensor-core pass: 16-column tiles per row
# 1, 2, 3-4, 5-8 and 9-64 (one to eight column groups of warps), rows not a multiple of
# 16, several row chunks, and systems that stream through the ring (above ~100 KB)
TC_SHAPES = [(5, 9), (16, 16), (17, 30), (40, 33), (33, 64), (70, 100), (100, 128), (130, 150), (64, 250),
             (200, 520), (600, 40), (300, 420), (257, 1024), (150, 600)]


@pytest.mark.parametrize("config", [STREAMED, TENSOR])
def test_bf16_two_steps_match_oracle_on_stored_matrix(tacta, config):
    """Two steps (t = 1, 2: every kind of pass -- Aᵀr alone, A z_i with Aᵀu_i, A z_t alone)
    with BF16 storage on CUDA cores and on the tensor cores, against the oracle run in FP64
    on the BF16-rounded matrix. The FP32 chain differs from it by FP32 rounding (about
    1e-7 relative per product, amplified by the 2 x 2 auxiliary solve), so x agrees to
    1e-4; a lost operand term (z or u carried in one or two BF16 terms, 2^-9 / 2^-17) or a
    misplaced fragment shows far above that."""
    rng = np.random.default_rng(11)
    mats = [rng.standard_normal(sh) for sh in TC_SHAPES]
    bs = [A @ rng.standard_normal(A.shape[1]) for A in mats]
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=2)
    xs, iters, rel, reason = run(tacta, mats, bs, tacta.BATCH_BF16, config=config, **opts)
    for s, (A, b) in enumerate(zip(mats, bs)):
        ref = oracle.cta_solve(oracle.make_operator(problem(bf16_round(A), b)), b, pivot_tol=1e-6, **opts)
        assert iters[s] == 2 and tacta.REASON[int(reason[s])] == "MAXITER", s
        err = np.linalg.norm(xs[s] - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-4, (s, A.shape, err)


def test_bf16_tensor_cores_one_step(tacta):
    """One step (t = 1: x = (phi_1 / phi_2) Aᵀ b) on the tensor cores against the oracle on
    the BF16-rounded matrix to 2e-5: the products' only error is FP32 accumulation."""
    rng = np.random.default_rng(12)
    mats = [rng.standard_normal(sh) for sh in TC_SHAPES]
    bs = [A @ rng.standard_normal(A.shape[1]) for A in mats]
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=1)
    xs, iters, rel, reason = run(tacta, mats, bs, tacta.BATCH_BF16, config=TENSOR, **opts)
    for s, (A, b) in enumerate(zip(mats, bs)):
        ref = oracle.cta_solve(oracle.make_operator(problem(bf16_round(A), b)), b, pivot_tol=1e-6, **opts)
        err = np.linalg.norm(xs[s] - ref.x) / np.linalg.norm(ref.x)
        assert err <= 2e-5, (s, A.shape, err)


def test_full_batch_4096_fp32(tacta):
    """The full workload: 4096 systems (m in [32, 512], n in [m/2, 2m], 10% rank m/2),
    FP32 storage, tol 1e-8, at most 20000 steps each. Every system that reports RESIDUAL
    has a host-recomputed FP64 residual within tol. The systems that are well conditioned
    by construction converge: full rank with n/m outside [0.8, 1.25] (Gaussian, condition
    number below ~20), and rank r = m/2 with n >= 1.5 r (U Vᵀ with both factors at least
    1.5 times as long as wide). Near-square systems (condition number up to ~1e3-1e4 at
    these sizes) may reach the step cap; at least 98% of all systems converge. Checked on
    the first solve (single blocks) and on the second, planned from the first's times,
    where thread-block clusters take the longest systems."""
    B0 = gen.dense_batch(4096, seed=7)
    B = tacta.Batch(B0.mats, storage=tacta.BATCH_FP32)
    opts = dict(tol=1e-8, tol_normal=0.0, max_iter=20000)
    for solve in range(2):
        if solve == 1:
            assert B.wide_plan(**opts)[0] > 0
        x, iters, rel, reason = B.cta(np.concatenate(B0.bs), **opts)
        x = B.split(x)
        names = [tacta.REASON[int(r)] for r in reason]
        for s, (A, b) in enumerate(zip(B0.mats, B0.bs)):
            m, n = A.shape
            assert names[s] in ("RESIDUAL", "MAXITER"), (solve, s, names[s])
            if names[s] == "RESIDUAL":
                r = np.linalg.norm(b - A @ x[s]) / np.linalg.norm(b)
                assert r <= 1e-8 * (1 + 1e-6), (solve, s, r)
                continue
            rank = m // 2 if B0.low_rank[s] else min(m, n)
            well = (n >= 1.5 * rank) if B0.low_rank[s] else (n / m >= 1.25 or n / m <= 0.8)
            assert not well, (solve, s, m, n, bool(B0.low_rank[s]), names[s], rel[s])
        assert names.count("RESIDUAL") >= 0.98 * len(names)
    B.close()


def test_timeline_and_stage_configs(tacta):
    """The batch timeline: every system of the last solve has a start and an end stamp on
    the device clock with end >= start; the fused-pass configurations report their ring
    stages (16/32/48 KB on CUDA cores, 40/48 KB on the tensor cores) and every
    configuration meets the tolerance on a BF16 batch."""
    mats, bs, _ = small_batch(8, 24, m_range=(40, 160), aspect=(1.4, 2.0))
    b = np.concatenate(bs)
    B = tacta.Batch(mats, storage=tacta.BATCH_BF16)
    x, iters, rel, reason = B.cta(b, tol=1e-8, tol_normal=0.0, max_iter=5000)
    tb, te = B.timeline()
    assert tb.shape == te.shape == (len(mats),)
    assert np.all(tb > 0) and np.all(te >= tb)
    stages = [c[2] for c in tacta.Batch.configs()]
    tc = tacta.Batch.tensor_core_configs()
    assert sorted(s for i, s in enumerate(stages) if s and i not in tc) == [16384, 32768, 49152]
    assert sorted(stages[i] for i in tc) == [40960, 49152]
    for c in range(len(stages)):
        B.set_config(c)
        _, _, rc, rs = B.cta(b, tol=1e-8, tol_normal=0.0, max_iter=5000)
        assert all(tacta.REASON[int(r)] == "RESIDUAL" for r in rs) and np.all(rc <= 1e-8 * (1 + 1e-6)), c
    B.close()


# ------------------------------------------------------------ thread-block clusters

def run_wide(tacta, mats, bs, storage, systems, cluster, clusters=0, **opts):
    B = tacta.Batch(mats, storage=storage)
    B.set_wide(systems, cluster, clusters)
    x, iters, rel, reason = B.cta(np.concatenate(bs), **opts)
    plan = B.wide_plan(**opts)
    xs = B.split(x)
    B.close()
    return xs, iters, rel, reason, plan


def wide_mix(seed):
    """Small systems (blocks of a C = 8 cluster with no rows at m < 8 ... 57), and large ones
    whose rows exceed a block's shared memory (read through L2)."""
    mats, bs, _ = small_batch(seed, 24, m_range=(5, 120))
    m2, b2, _ = small_batch(seed + 100, 6, m_range=(300, 512))
    return mats + m2, bs + b2


@pytest.mark.parametrize("cluster", [2, 4, 8, 16])
def test_wide_fp64_fixed_trajectories_match_oracle(tacta, cluster):
    """Every system on a cluster (FP64 storage, four steps t = 1..4 each): x, the step
    count and the recomputed residual against the oracle's run on that system alone, as
    for one block; fewer clusters than systems, so clusters take several in turn."""
    mats, bs = wide_mix(21)
    opts = dict(tol=1e-30, tol_normal=0.0, max_iter=4)
    xs, iters, rel, reason, plan = run_wide(tacta, mats, bs, tacta.BATCH_FP64, len(mats), cluster, 5, **opts)
    assert plan[:3] == (len(mats), cluster, 5)
    for s, (A, b) in enumerate(zip(mats, bs)):
        ref = oracle.cta_solve(oracle.make_operator(problem(A, b)), b, **opts)
        assert iters[s] == ref.iters, s
        assert np.linalg.norm(xs[s] - ref.x) <= 1e-9 * np.linalg.norm(ref.x), (s, A.shape)
        assert rel[s] == pytest.approx(ref.rel_res, rel=1e-9), s
        assert tacta.REASON[int(reason[s])] == "MAXITER"


@pytest.mark.parametrize("storage,tol,xtol", [("BATCH_FP64", 1e-10, 1e-8), ("BATCH_FP32", 1e-8, 1e-6),
                                              ("BATCH_BF16", 1e-8, 3e-2)])
@pytest.mark.parametrize("cluster,share", [(16, 0.5), (8, 1.0), (4, 0.5), (2, 0.25)])
def test_wide_to_tolerance_min_norm(tacta, storage, tol, xtol, cluster, share):
    """Clusters on all, half or a quarter of the systems (the rest on single blocks of the
    dependent launch at the same time), each precision: the host-recomputed FP64 residual
    meets tol, the reported one equals it, x is the minimum-norm solution within cond(A)
    times xtol, and with every system on a cluster a second solve gives the same bits."""
    mats, bs, _ = small_batch(2, 40, aspect=(1.4, 2.0))
    m2, b2, _ = small_batch(6, 8, m_range=(220, 400), aspect=(1.4, 1.8))
    mats, bs = m2 + mats, b2 + bs
    k = max(1, int(share * len(mats)))
    B = tacta.Batch(mats, storage=getattr(tacta, storage))
    B.set_wide(k, cluster)
    opts = dict(tol=tol, tol_normal=0.0, max_iter=20000)
    x, iters, rel, reason = B.cta(np.concatenate(bs), **opts)
    x2, iters2, _, _ = B.cta(np.concatenate(bs), **opts)
    if k == len(mats):   # (with fewer, the learned order may move other systems to the head)
        assert np.array_equal(x, x2) and np.array_equal(iters, iters2)
    assert B.wide_plan(**opts)[:2] == (k, cluster)
    xs = B.split(x)
    B.close()
    for s, (A, b) in enumerate(zip(mats, bs)):
        assert tacta.REASON[int(reason[s])] == "RESIDUAL", (s, reason[s], rel[s])
        r = np.linalg.norm(b - A @ xs[s]) / np.linalg.norm(b)
        assert r <= tol * (1 + 1e-6), (s, r)
        assert rel[s] == pytest.approx(r, rel=1e-6, abs=1e-14)
        sv = np.linalg.svd(A, compute_uv=False)
        sv = sv[sv > 1e-10 * sv[0]]
        xmn = np.linalg.pinv(A, rcond=1e-10) @ b
        err = np.linalg.norm(xs[s] - xmn) / np.linalg.norm(xmn)
        assert err <= xtol * sv[0] / sv[-1], (s, err)


@pytest.mark.parametrize("cluster", [8, 16])
def test_wide_edge_cases(tacta, cluster):
    """On clusters of 8 and 16: 1 x 1, one row, one column (blocks without rows or columns),
    a zero right-hand side, and max_iter = 0."""
    rng = np.random.default_rng(3)
    mats = [np.array([[2.0]]), rng.standard_normal((1, 7)), rng.standard_normal((9, 1)),
            rng.standard_normal((30, 40))]
    bs = [np.array([4.0]), rng.standard_normal(1), mats[2] @ np.array([1.5]), np.zeros(30)]
    xs, iters, rel, reason, _ = run_wide(tacta, mats, bs, tacta.BATCH_FP64, 4, cluster, tol=1e-12,
                                         tol_normal=0.0, max_iter=1000)
    assert xs[0][0] == pytest.approx(2.0, rel=1e-14)
    np.testing.assert_allclose(xs[1], np.linalg.pinv(mats[1]) @ bs[1], rtol=1e-10, atol=1e-12)
    assert xs[2][0] == pytest.approx(1.5, rel=1e-10)
    assert tacta.REASON[int(reason[3])] == "ZERO_RHS" and np.all(xs[3] == 0.0) and iters[3] == 0
    xs, iters, rel, reason, _ = run_wide(tacta, mats[:3], bs[:3], tacta.BATCH_FP32, 3, cluster, tol=1e-8,
                                         tol_normal=0.0, max_iter=0)
    assert all(tacta.REASON[int(r)] == "MAXITER" for r in reason)
    assert np.all(iters == 0) and np.allclose(rel, 1.0) and all(np.all(x == 0.0) for x in xs)


def test_wide_normal_equation_stop(tacta):
    """The normal-equation test (||Aᵀr|| <= tol_normal ||Aᵀb||) on a cluster: an
    inconsistent overdetermined system stops with reason NORMAL at the least-squares
    solution, as on one block."""
    rng = np.random.default_rng(17)
    A = rng.standard_normal((200, 60))
    b = rng.standard_normal(200)
    opts = dict(tol=1e-12, tol_normal=1e-9, max_iter=20000)
    xs, iters, rel, reason, _ = run_wide(tacta, [A], [b], tacta.BATCH_FP64, 1, 4, **opts)
    xs1, iters1, _, reason1 = run(tacta, [A], [b], tacta.BATCH_FP64, **opts)
    xls = np.linalg.lstsq(A, b, rcond=None)[0]
    assert tacta.REASON[int(reason[0])] == "NORMAL" == tacta.REASON[int(reason1[0])]
    assert np.linalg.norm(xs[0] - xls) <= 1e-6 * np.linalg.norm(xls)
    assert np.linalg.norm(xs1[0] - xls) <= 1e-6 * np.linalg.norm(xls)


def test_wide_plan_automatic(tacta):
    """The planner: no clusters before any solve; after one, on a batch whose few
    near-square systems take far longer than the rest, it puts the longest on clusters
    with a smaller predicted makespan than one block each, and the solves meet the
    tolerance wherever the systems converge."""
    rng = np.random.default_rng(5)
    mats, bs = [], []
    for s in range(600):
        m = int(rng.integers(32, 96))
        n = int(2 * m)
        mats.append(rng.standard_normal((m, n)))
    for s in range(4):   # near-square: thousands of steps
        mats.append(rng.standard_normal((400, 400)))
    bs = [A @ rng.standard_normal(A.shape[1]) for A in mats]
    b = np.concatenate(bs)
    B = tacta.Batch(mats, storage=tacta.BATCH_FP32)
    opts = dict(tol=1e-8, tol_normal=0.0, max_iter=3000)
    assert B.wide_plan(**opts) == (0, 0, 0, 0.0)
    B.cta(b, **opts)
    systems, cluster, clusters, ms = B.wide_plan(**opts)
    B.set_wide(0)
    ms_off = B.wide_plan(**opts)[3]
    B.set_wide(-1)
    assert systems >= 1 and cluster in (2, 4, 8, 16) and 1 <= clusters <= systems
    assert 0 < ms < ms_off
    for _ in range(2):
        x, iters, rel, reason = B.cta(b, **opts)
        xs = B.split(x)
        for s, (A, bb) in enumerate(zip(mats, bs)):
            if tacta.REASON[int(reason[s])] == "RESIDUAL":
                assert np.linalg.norm(bb - A @ xs[s]) / np.linalg.norm(bb) <= 1e-8 * (1 + 1e-6), s
            else:
                assert tacta.REASON[int(reason[s])] == "MAXITER" and A.shape == (400, 400), s
    B.close()
