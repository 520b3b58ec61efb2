"""Seeded synthetic inputs for the TA / CTA solvers.

This module only *builds problems* (matrices, right-hand sides and known
solutions). It holds none of the solvers' arithmetic: no residual updates, no
Krylov chains, no step sizes. Both the CPU oracle and the CUDA path are fed
from here, so that the two sides see byte-identical inputs.

Right-hand sides follow the paper's convention b = A·x_known (Sec. 5: b is the
row-sum vector, i.e. x_known = 1, for square systems and for the rectangular
lpnetlib runs). The product A·x_known is formed with scipy.sparse / numpy
(library routines), never with solver code.

Shapes and structure follow the paper's workloads:
  * dense Gaussian square systems and a low-rank variant (min-norm target),
  * the 2D convection-diffusion 5-point stencil (the paper's MVMMCD CFD family,
    Sec. 5.1) on an N x N grid,
  * the Clement tridiagonal matrix (Sec. 5.1, Clement tables),
  * an LP-like rectangular m << n sparse matrix with duplicated scaled rows
    (stand-in for the lpnetlib set of Sec. 5.2, which is not available here),
  * small ragged / empty-row CSR matrices for edge cases,
  * batches of uneven dense systems (m in [32, 512], n in [m/2, 2m], 10% of rank
    m/2) for the batched solver.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Problem", "dense_gaussian", "dense_low_rank", "convdiff_stencil",
    "clement", "lp_rect", "random_csr", "diag_matrix", "DenseBatch", "dense_batch", "banded_rect",
]


@dataclass
class Problem:
    """A linear system A x = b with A dense row-major or CSR (int32 indices)."""
    name: str
    m: int
    n: int
    fmt: str                      # "dense" or "csr"
    dense: np.ndarray | None = None        # (m, n) float64, C order
    rowptr: np.ndarray | None = None       # (m+1,) int32
    colidx: np.ndarray | None = None       # (nnz,) int32
    vals: np.ndarray | None = None         # (nnz,) float64
    b: np.ndarray | None = None            # (m,) float64
    x_known: np.ndarray | None = None      # the x used to build b (not necessarily min-norm)
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.m * self.n) if self.fmt == "dense" else int(self.vals.size)

    def scipy(self) -> sp.csr_matrix:
        """The matrix as scipy CSR (for building inputs and for pins)."""
        if self.fmt == "dense":
            return sp.csr_matrix(self.dense)
        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.m, self.n))

    def to_dense(self) -> np.ndarray:
        if self.fmt == "dense":
            return self.dense
        return self.scipy().toarray()

    def as_csr(self) -> "Problem":
        """The same system in CSR storage (dense input converted, zeros dropped)."""
        if self.fmt == "csr":
            return self
        S = sp.csr_matrix(self.dense)
        S.sort_indices()
        return Problem(self.name + "_csr", self.m, self.n, "csr", None,
                       S.indptr.astype(np.int32), S.indices.astype(np.int32),
                       S.data.astype(np.float64), self.b, self.x_known, dict(self.meta))

    def as_dense(self) -> "Problem":
        if self.fmt == "dense":
            return self
        return Problem(self.name + "_dense", self.m, self.n, "dense",
                       np.ascontiguousarray(self.to_dense()), b=self.b,
                       x_known=self.x_known, meta=dict(self.meta))


def _from_scipy(name, S, x_known, meta=None) -> Problem:
    S = sp.csr_matrix(S)
    S.sum_duplicates()
    S.sort_indices()
    m, n = S.shape
    b = np.asarray(S @ x_known, dtype=np.float64)
    return Problem(name, m, n, "csr", None,
                   np.ascontiguousarray(S.indptr, dtype=np.int32),
                   np.ascontiguousarray(S.indices, dtype=np.int32),
                   np.ascontiguousarray(S.data, dtype=np.float64),
                   b, np.asarray(x_known, dtype=np.float64), meta or {})


def dense_gaussian(m: int = 256, n: int = 256, seed: int = 0) -> Problem:
    """A_ij ~ N(0,1), x_known ~ N(0,1) from the same stream, b = A x_known."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    x = rng.standard_normal(n)
    return Problem(f"dense_gauss_{m}x{n}_s{seed}", m, n, "dense", np.ascontiguousarray(A),
                   b=A @ x, x_known=x, meta={"seed": seed})


def dense_low_rank(m: int = 256, n: int = 256, rank: int = 128, seed: int = 1) -> Problem:
    """A = U V^T with U (m x rank), V (n x rank) ~ N(0,1); b = A x_known, x_known ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((n, rank))
    A = U @ V.T
    x = rng.standard_normal(n)
    return Problem(f"dense_rank{rank}_{m}x{n}_s{seed}", m, n, "dense", np.ascontiguousarray(A),
                   b=A @ x, x_known=x, meta={"seed": seed, "rank": rank})


def convdiff_stencil(N: int = 1000, peclet: float = 0.5, velocity=(1.0, 0.5)) -> Problem:
    """2D convection-diffusion -Δu + β·∇u on the unit square, Dirichlet boundary,
    central 5-point differences on an N x N interior grid, scaled by h².

    Unknown (i, j) (i = x index fastest) is row j*N + i. Diffusion is 1; β is
    `velocity` scaled so the cell Péclet number max_k |β_k| h / 2 equals
    `peclet`. Row entries: centre 4, west -1-β_x h/2, east -1+β_x h/2,
    south -1-β_y h/2, north -1+β_y h/2. b = A·1 (x_known = 1).
    """
    vx, vy = velocity
    scale = 2.0 * peclet / max(abs(vx), abs(vy))   # β h = scale * velocity
    bxh, byh = scale * vx, scale * vy
    w, e = -1.0 - bxh / 2, -1.0 + bxh / 2
    s_, nn = -1.0 - byh / 2, -1.0 + byh / 2
    I = sp.identity(N, format="csr")
    Tx = sp.diags([np.full(N - 1, w), np.full(N, 4.0), np.full(N - 1, e)], [-1, 0, 1], format="csr")
    Ty = sp.diags([np.full(N - 1, s_), np.full(N - 1, nn)], [-1, 1], format="csr")
    A = sp.kron(I, Tx, format="csr") + sp.kron(Ty, I, format="csr")
    return _from_scipy(f"convdiff_{N}x{N}", A, np.ones(N * N),
                       {"N": N, "coef": {"C": 4.0, "W": w, "E": e, "S": s_, "Nn": nn}})


def clement(n: int = 100001) -> Problem:
    """Clement tridiagonal matrix: A[i,i+1] = A[i+1,i] = sqrt(i (n-i)) (1-based i),
    zero diagonal. Singular for odd n. b = A·1, which lies in range(A)."""
    i = np.arange(1, n, dtype=np.float64)
    c = np.sqrt(i * (n - i))
    A = sp.diags([c, c], [-1, 1], shape=(n, n), format="csr")
    return _from_scipy(f"clement_{n}", A, np.ones(n), {"n": n})


def lp_rect(m: int = 10000, n: int = 1_000_000, per_col: int = 30, dup_rows: int = 500,
            x_density: float = 0.01, seed: int = 3) -> Problem:
    """LP-like underdetermined sparse matrix (m << n), rank-deficient.

    m - dup_rows base rows; every column gets `per_col` nonzeros at distinct
    uniform-random base rows with values U(-1, 1). Then `dup_rows` extra rows
    are copies of distinct random base rows, each scaled by U(0.5, 2). Rows are
    shuffled. x_known has `x_density` nonzeros ~ N(0,1); b = A x_known
    (consistent; the min-norm solution is A⁺b, not x_known).
    """
    rng = np.random.default_rng(seed)
    mb = m - dup_rows
    k = min(per_col, mb)
    rows = rng.integers(0, mb, size=(n, k))
    # resample columns that drew a repeated row until every column is distinct
    while True:
        srt = np.sort(rows, axis=1)
        bad = np.any(srt[:, 1:] == srt[:, :-1], axis=1) if k > 1 else np.zeros(n, bool)
        if not bad.any():
            break
        rows[bad] = rng.integers(0, mb, size=(int(bad.sum()), k))
    rows = np.sort(rows, axis=1)
    vals = rng.uniform(-1.0, 1.0, size=(n, k))
    cols = np.repeat(np.arange(n), k)
    base = sp.csr_matrix((vals.ravel(), (rows.ravel(), cols)), shape=(mb, n))
    sel = rng.choice(mb, size=dup_rows, replace=False)
    scl = rng.uniform(0.5, 2.0, size=dup_rows)
    extra = sp.diags(scl) @ base[sel]
    A = sp.vstack([base, extra], format="csr")
    perm = rng.permutation(m)
    A = A[perm]
    x = np.zeros(n)
    nzx = rng.choice(n, size=max(1, int(round(x_density * n))), replace=False)
    x[nzx] = rng.standard_normal(nzx.size)
    return _from_scipy(f"lp_rect_{m}x{n}", A, x, {"seed": seed, "per_col": per_col,
                                                 "dup_rows": dup_rows})


def banded_rect(m: int, n: int, offsets=(0, 1, 3), seed: int = 3) -> Problem:
    """A well-conditioned banded m x n matrix (m <= n): the main diagonal U(1.5, 2.5), the
    other diagonals col - row = offset U(-0.4, 0.4) (diagonally dominant rows, so full row
    rank with singular values in ~[0.7, 3.3]); x_known ~ N(0,1), b = A x_known, which
    has a component in the null space of A when m < n (x_known is not the minimum-norm
    solution). Its minimum-norm problems make Algorithm 2.5's trips short."""
    rng = np.random.default_rng(seed)
    diags = [rng.uniform(1.5, 2.5, min(m, n - k)) if k == 0 else rng.uniform(-0.4, 0.4, min(m, n - k))
             for k in offsets]
    S = sp.diags(diags, list(offsets), shape=(m, n), format="csr")
    x = np.random.default_rng(seed + 1).standard_normal(n)
    return _from_scipy(f"banded_{m}x{n}", S, x, {"offsets": list(offsets)})


def random_csr(m: int, n: int, density: float = 0.05, seed: int = 0, empty_rows: int = 0,
               long_rows: int = 0, long_len: int | None = None, x_known=None) -> Problem:
    """Random CSR with ragged rows: optional all-zero rows and a few long rows."""
    rng = np.random.default_rng(seed)
    S = sp.random(m, n, density=density, format="lil", random_state=rng,
                  data_rvs=lambda s: rng.uniform(-1.0, 1.0, s))
    if long_rows:
        L = long_len or n
        for r in rng.choice(m, size=min(long_rows, m), replace=False):
            cols = rng.choice(n, size=min(L, n), replace=False)
            S[r, cols] = rng.uniform(-1.0, 1.0, cols.size)
    S = sp.csr_matrix(S)
    if empty_rows:
        er = rng.choice(m, size=min(empty_rows, m), replace=False)
        mask = np.ones(m)
        mask[er] = 0.0
        S = sp.csr_matrix(sp.diags(mask) @ S)
        S.eliminate_zeros()
    if x_known is None:
        x_known = rng.standard_normal(n)
    return _from_scipy(f"random_csr_{m}x{n}_s{seed}", S, x_known, {"seed": seed})


def diag_matrix(d: np.ndarray, x_known=None) -> Problem:
    """Diagonal CSR matrix diag(d) (the paper's PD / PSD / indefinite diagonal
    families); b = A·1 unless x_known is given. Zero diagonal entries are kept
    out of the storage."""
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    A = sp.diags(d, 0, shape=(n, n), format="csr")
    A.eliminate_zeros()
    return _from_scipy(f"diag_{n}", A, np.ones(n) if x_known is None else x_known)


@dataclass
class DenseBatch:
    """Independent dense systems A_s x = b_s, b_s = A_s x*_s (consistent)."""
    mats: list                     # A_s, (m_s, n_s) float64 C order
    bs: list                       # b_s
    xstar: list                    # x*_s
    low_rank: np.ndarray           # bool per system: A_s = U V^T of rank m_s / 2

    @property
    def count(self) -> int:
        return len(self.mats)

    def packed_b(self) -> np.ndarray:
        return np.concatenate(self.bs) if self.bs else np.zeros(0)


def dense_batch(count: int = 4096, m_range=(32, 512), low_rank_frac: float = 0.1,
                seed: int = 7) -> DenseBatch:
    """Uneven dense systems: m uniform in m_range, n uniform in [ceil(m/2), 2m], entries
    N(0,1); a fraction low_rank_frac is U V^T of rank floor(m/2) (U, V Gaussian, scaled to
    unit-variance entries); b = A x* with x* ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    mats, bs, xs = [], [], []
    lr = np.zeros(count, dtype=bool)
    for s in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers((m + 1) // 2, 2 * m + 1))
        if rng.random() < low_rank_frac:
            r = max(1, m // 2)
            A = (rng.standard_normal((m, r)) @ rng.standard_normal((r, n))) / np.sqrt(r)
            lr[s] = True
        else:
            A = rng.standard_normal((m, n))
        x = rng.standard_normal(n)
        mats.append(np.ascontiguousarray(A))
        xs.append(x)
        bs.append(A @ x)
    return DenseBatch(mats=mats, bs=bs, xstar=xs, low_rank=lr)
