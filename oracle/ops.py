"""Matrix-vector products for the oracle (test infrastructure only).

A is m x n, stored dense row-major or CSR (rowptr int32 m+1, colidx int32,
vals float64). The products are the definitions:

    (A x)_i   = sum_{k = rowptr[i]}^{rowptr[i+1]-1} vals[k] * x[colidx[k]]
    (Aᵀ r)_j = sum over nonzeros k in column j of vals[k] * r[row(k)]

written as a weighted bincount over the nonzeros (each output sums its terms
in nonzero order). Dense products use numpy's matmul.

``NormalOperator`` is the implicit operator AᵀA used when TA runs on the
normal equation (Sec. 5.2: "the inputs for TA are AᵀA and Aᵀb, used implicitly
via matrix-vector multiplications").
"""
from __future__ import annotations

import numpy as np


class Operator:
    """y = A x and z = Aᵀ r for a dense or CSR matrix, counting products."""

    def __init__(self, m, n, fmt, dense=None, rowptr=None, colidx=None, vals=None):
        self.m, self.n, self.fmt = int(m), int(n), fmt
        self.nmatvec = 0
        if fmt == "dense":
            self.A = np.asarray(dense, dtype=np.float64).reshape(self.m, self.n)
        elif fmt == "csr":
            self.rowptr = np.asarray(rowptr, dtype=np.int64)
            self.colidx = np.asarray(colidx, dtype=np.int64)
            self.vals = np.asarray(vals, dtype=np.float64)
            # row index of every stored nonzero
            self.row_of = np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.rowptr))
        else:
            raise ValueError(f"unknown format {fmt!r}")

    def matvec(self, x):
        """A x."""
        self.nmatvec += 1
        x = np.asarray(x, dtype=np.float64)
        if self.fmt == "dense":
            return self.A @ x
        return np.bincount(self.row_of, weights=self.vals * x[self.colidx], minlength=self.m)

    def rmatvec(self, r):
        """Aᵀ r."""
        self.nmatvec += 1
        r = np.asarray(r, dtype=np.float64)
        if self.fmt == "dense":
            return self.A.T @ r
        return np.bincount(self.colidx, weights=self.vals * r[self.row_of], minlength=self.n)


class NormalOperator:
    """The n x n operator M = AᵀA, applied as Aᵀ(A x); symmetric, so Mᵀ = M."""

    def __init__(self, A: Operator):
        self.A = A
        self.m = self.n = A.n
        self.fmt = "normal"

    @property
    def nmatvec(self):
        return self.A.nmatvec

    def matvec(self, x):
        return self.A.rmatvec(self.A.matvec(x))

    def rmatvec(self, r):
        return self.A.rmatvec(self.A.matvec(r))


def make_operator(p) -> Operator:
    """Operator from any object with the attributes of ``gen.Problem``."""
    if p.fmt == "dense":
        return Operator(p.m, p.n, "dense", dense=p.dense)
    return Operator(p.m, p.n, "csr", rowptr=p.rowptr, colidx=p.colidx, vals=p.vals)
