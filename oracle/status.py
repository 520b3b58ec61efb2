"""Outcome codes of the oracle solvers (test infrastructure only).

``Status`` says whether the call produced an answer; ``Reason`` says which
stopping rule ended the iteration (Alg. 1.1 while-clauses, Alg. 2.1/2.2/2.5
while-clauses and the witness STOP).
"""
from enum import IntEnum


class Status(IntEnum):
    OK = 0          # a stopping test of the algorithm was met
    MAXITER = 1     # iteration cap reached first
    BREAKDOWN = 2   # the step is undefined (zero Hankel rank, zero ||v - b'||)
    WITNESS = 3     # Alg. 2.1 stopped on a witness (b not in E_{A,rho})
    NONFINITE = -2  # a NaN / Inf appeared in a reduction


class Reason(IntEnum):
    NONE = 0
    RESIDUAL = 1    # ||b - A x|| <= tol ||b||
    NORMAL = 2      # ||A^T (b - A x)|| <= tol_normal ||A^T b||
    MAXITER = 3
    BREAKDOWN = 4
    WITNESS = 5
    GAP = 6         # Alg. 2.5: rho_upper - rho_lower <= gap tolerance
    ZERO_RHS = 7    # b = 0: x = 0 is the minimum-norm solution
    NONFINITE = 8
    RHO_BOUND = 10  # TA with x >= 0 (Sec. 6): rho passed its termination bound
    ENHANCED = 11   # enhanced CTA (Sec. 3.2): a first-order iterate met the normal-equation test
