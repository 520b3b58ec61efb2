"""CTA with the columns of A spread over several GPUs, one process per GPU.

Alg. 1.1 with H = A Aᵀ (Sec. 3, Sec. 5): split A = [A_1 ... A_G] by columns (the
balanced split of tacta_column_partition), so H = sum_g A_g A_gᵀ. Every rank keeps its
slice x_g of x and the replicated m-vectors r, u_i; per H-apply

    z_{i,g} = A_gᵀ u_{i-1}                      local product with the slice
    [A_g z_{i,g} | ||z_{i,g}||² | 0]            one all-reduce (sum) of m + 2 doubles
    u_i = sum_g A_g z_{i,g},  phi_{2i-1} = sum_g ||z_{i,g}||²,  phi_{2i} = ||u_i||²

The all-reduce hands every rank the same sums, so every rank solves the same auxiliary
equation (tacta_aux_solve, the code the single-GPU kernels run) on the same bits, and
updates x_g += sum alpha_i z_{i,g} and r -= sum alpha_i u_i. The true residual
b - sum_g A_g x_g (every recompute_every steps, and before a stop on the residual test)
takes one more all-reduce of the same layout. The stop tests are those of the
single-GPU solver: ||r|| <= tol ||b|| on the true residual, ||Aᵀ r|| <= tol_normal
||Aᵀ b|| (phi_1), the iteration cap.

The products run through the library (a Plan of the slice on the rank's GPU); the
communicator is torch.distributed (NCCL on GPUs). The same driver runs on CPU tensors
with the gloo backend and a CPU stand-in for the slice's products, which is how its
partition and reduction bookkeeping is tested in this repository (one GPU per machine
here: the multi-GPU path is not measured).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import aux_solve, column_partition

__all__ = ["column_slice", "PlanShard", "ShardResult", "sharded_cta", "PAYLOAD_EXTRA"]

PAYLOAD_EXTRA = 2   # doubles after the m-vector in an all-reduce buffer: the norm partial, a zero pad


def column_slice(rowptr, colidx, vals, m, c0, c1):
    """Host CSR arrays of A[:, c0:c1] (columns renumbered from 0)."""
    rowptr = np.asarray(rowptr)
    colidx = np.asarray(colidx)
    vals = np.asarray(vals)
    keep = (colidx >= c0) & (colidx < c1)
    counts = np.add.reduceat(keep.astype(np.int64), rowptr[:-1]) if colidx.size else np.zeros(m, np.int64)
    counts[np.diff(rowptr) == 0] = 0
    rp = np.zeros(m + 1, dtype=np.int32)
    np.cumsum(counts, out=rp[1:])
    return rp, (colidx[keep] - c0).astype(np.int32), vals[keep].astype(np.float64)


class PlanShard:
    """The slice A_g (m x n_g) on this rank's GPU: products through a tacta Plan."""

    def __init__(self, plan, m, n_local):
        self.plan, self.m, self.n_local = plan, m, n_local

    def matvec(self, z):          # A_g z (m)
        return self.plan.matvec(z)

    def rmatvec(self, u):         # A_gᵀ u (n_g)
        return self.plan.matvec(u, transpose=True)


@dataclass
class ShardResult:
    x: object                     # this rank's slice x_g
    reason: str
    iters: int
    rel_res: float
    hist: list = field(default_factory=list)     # ||r|| / ||b|| after each step (hist[0] at the start)
    trace: list = field(default_factory=list)    # per step: (t, phi_1..phi_2t, alpha)


def _schedule(k, t_max, cycle):
    """t of step k (Sec. 5.1: ping-pong 1..t_max..1; 1 = sawtooth, 2 = fixed t_max)."""
    if cycle == 2 or t_max == 1:
        return t_max
    if cycle == 1:
        return 1 + k % t_max
    period = 2 * t_max - 2
    j = k % period
    return j + 1 if j < t_max else 2 * t_max - 1 - j


def sharded_cta(op, b, dist, tol=1e-10, tol_normal=None, max_iter=1000, t_max=5, cycle=0,
                recompute_every=40, pivot_tol=1e-12, keep_trace=False) -> ShardResult:
    """CTA from x = 0 on the column-sharded operator `op` (matvec: A_g z -> m-vector,
    rmatvec: A_gᵀ u -> n_g-vector, both torch tensors of b's device) with the
    torch.distributed process group `dist`. b: the replicated right-hand side."""
    import torch
    if tol_normal is None or tol_normal < 0:
        tol_normal = tol
    m = op.m

    def allreduce(vec, scal):
        buf = torch.cat([vec, torch.tensor([scal, 0.0], dtype=vec.dtype, device=vec.device)])
        dist.all_reduce(buf)
        return buf[:m], float(buf[m])

    def dot(a, c):
        return float(torch.dot(a, c))

    def true_residual(x):
        ax, _ = allreduce(op.matvec(x), 0.0)
        r = b - ax
        return r, dot(r, r)

    bn2 = dot(b, b)
    if bn2 == 0.0:
        return ShardResult(torch.zeros(op.n_local, dtype=b.dtype, device=b.device), "ZERO_RHS", 0, 0.0)
    atb = op.rmatvec(b)
    z0 = torch.zeros(m, dtype=b.dtype, device=b.device)
    _, mtbn2 = allreduce(z0, dot(atb, atb))
    res_thr, nrm_thr = tol * tol * bn2, tol_normal * tol_normal * mtbn2
    x = torch.zeros(op.n_local, dtype=b.dtype, device=b.device)
    r, rn2, is_true, k = b.clone(), bn2, True, 0
    hist, trace = [math.sqrt(rn2 / bn2)], []
    reason = "MAXITER"
    while True:
        # the tests at the top of the loop: a passing recursive residual is checked on the true one
        if rn2 <= res_thr:
            if is_true:
                reason = "RESIDUAL"
                break
            r, rn2 = true_residual(x)
            is_true = True
            hist[-1] = math.sqrt(rn2 / bn2)
            continue
        if k >= max_iter:
            break
        t = _schedule(k, t_max, cycle)
        phi = np.zeros(2 * t + 1)
        zs, us = [], []
        u = r
        for i in range(1, t + 1):
            z = op.rmatvec(u)
            u, phi[2 * i - 1] = allreduce(op.matvec(z), dot(z, z))
            phi[2 * i] = dot(u, u)
            zs.append(z)
            us.append(u)
        if not np.all(np.isfinite(phi[1:])):
            reason = "NONFINITE"
            break
        if phi[1] <= nrm_thr:
            reason = "NORMAL"
            break
        alpha, rank = aux_solve(phi, t, pivot_tol)
        if rank == 0:
            reason = "BREAKDOWN"
            break
        for a, z, uu in zip(alpha, zs, us):
            x = x + float(a) * z
            r = r - float(a) * uu
        rn2, is_true, k = dot(r, r), False, k + 1
        if keep_trace:
            trace.append((t, phi.copy(), np.array(alpha)))
        if recompute_every > 0 and k % recompute_every == 0:
            r, rn2 = true_residual(x)
            is_true = True
        hist.append(math.sqrt(rn2 / bn2))
    _, rt2 = true_residual(x)
    return ShardResult(x, reason, k, math.sqrt(rt2 / bn2), hist, trace)
