"""The column-sharded CTA (paper_2304_12168_gb300.sharded) with two gloo ranks on CPU.

Each rank takes its column slice from tacta_column_partition (the library's host entry
point), runs the sharded driver with the one all-reduce per H-apply, and the pieces are
checked against the unsharded computation: the first step's u_1 and moments (1e-14:
only the order of the sum over the shards differs), the gathered x after 8 steps
against the oracle (1e-9, the FP64 parity tolerance), and a run to tolerance on a
consistent system against the oracle's answer. The slices' products run on the host
here (scipy); on GPUs the same driver takes a library Plan per slice and NCCL.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import gen


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    return gen.lp_rect(m=300, n=2400, per_col=6, dup_rows=20, x_density=0.05, seed=5)


class _HostShard:
    """CPU stand-in for a slice's products (scipy), with the driver's torch interface."""

    def __init__(self, S):
        self.S, self.St = S, S.T.tocsr()
        self.m, self.n_local = S.shape

    def matvec(self, z):
        import torch
        return torch.from_numpy(self.S @ z.numpy())

    def rmatvec(self, u):
        import torch
        return torch.from_numpy(self.St @ u.numpy())


def _worker(rank, world, port, out):
    import scipy.sparse as sp
    import torch
    import torch.distributed as dist
    import paper_2304_12168_gb300 as tacta
    from paper_2304_12168_gb300.sharded import column_slice, sharded_cta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _problem()
    cb, snnz = tacta.column_partition(p.rowptr, p.colidx, p.m, p.n, world)
    c0, c1 = int(cb[rank]), int(cb[rank + 1])
    rp, ci, va = column_slice(p.rowptr, p.colidx, p.vals, p.m, c0, c1)
    op = _HostShard(sp.csr_matrix((va, ci, rp), shape=(p.m, c1 - c0)))
    b = torch.from_numpy(p.b.copy())
    res = sharded_cta(op, b, dist, tol=1e-30, tol_normal=0.0, max_iter=8, keep_trace=True)
    res2 = sharded_cta(op, b, dist, tol=1e-10, tol_normal=0.0, max_iter=5000)
    out[rank] = dict(cb=cb.tolist(), snnz=snnz.tolist(), x=res.x.numpy(), trace=res.trace, iters=res.iters,
                     reason=res.reason, x2=res2.x.numpy(), iters2=res2.iters, reason2=res2.reason,
                     rel2=res2.rel_res, hist=res.hist)
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0
    return dict(out)


def test_partition_is_balanced_and_covers_the_columns(two_ranks):
    p = _problem()
    cb = np.array(two_ranks[0]["cb"])
    assert cb[0] == 0 and cb[-1] == p.n and np.all(np.diff(cb) >= 1)
    counts = np.bincount(p.colidx, minlength=p.n)
    snnz = np.array(two_ranks[0]["snnz"])
    assert snnz.sum() == p.nnz
    assert np.all(snnz == [counts[cb[g]:cb[g + 1]].sum() for g in range(2)])
    assert snnz.max() - snnz.min() <= 2 * counts.max()      # split within a column of the ideal
    assert two_ranks[1]["cb"] == two_ranks[0]["cb"]


def test_first_h_apply_matches_the_unsharded_products(two_ranks):
    """u_1 = A Aᵀ b and the moments of the first F_1 step (phi_1 = ||Aᵀ b||²,
    phi_2 = ||A Aᵀ b||²) against products with the whole matrix."""
    p = _problem()
    S = p.scipy()
    z = S.T @ p.b
    u = S @ z
    t, phi, alpha = two_ranks[0]["trace"][0]
    assert t == 1
    assert phi[1] == pytest.approx(float(z @ z), rel=1e-14)
    assert phi[2] == pytest.approx(float(u @ u), rel=1e-14)
    # the same bits on both ranks (the all-reduce hands both the same sums)
    for (t0, ph0, al0), (t1, ph1, al1) in zip(two_ranks[0]["trace"], two_ranks[1]["trace"]):
        assert t0 == t1 and np.array_equal(ph0, ph1) and np.array_equal(al0, al1)


def test_eight_steps_match_the_oracle(two_ranks):
    import oracle
    p = _problem()
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-30, tol_normal=0.0, max_iter=8)
    x = np.concatenate([two_ranks[0]["x"], two_ranks[1]["x"]])
    assert two_ranks[0]["iters"] == ref.iters == 8
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    np.testing.assert_allclose(two_ranks[0]["hist"], ref.hist, rtol=1e-9)


def test_run_to_tolerance_matches_the_oracle(two_ranks):
    import oracle
    p = _problem()
    ref = oracle.cta_solve(oracle.make_operator(p), p.b, tol=1e-10, tol_normal=0.0, max_iter=5000)
    x = np.concatenate([two_ranks[0]["x2"], two_ranks[1]["x2"]])
    assert two_ranks[0]["reason2"] == "RESIDUAL" and two_ranks[0]["rel2"] <= 1e-10
    assert abs(two_ranks[0]["iters2"] - ref.iters) <= 1
    assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
