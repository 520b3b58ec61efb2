"""FP64 CPU oracle for the Triangle Algorithm (TA) and the Centering Triangle
Algorithm (CTA) of Lau & Kalantari, arXiv:2304.12168.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain, obviously correct
statement of what the CUDA solvers compute. Only the test suite, the smoke
check in ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it. The product path (``paper_2304_12168_gb300``) never imports,
links or calls anything here, and this package never imports the product.

Everything is numpy float64. Matrix-vector products are written as their
definitions (dense: a BLAS matmul; CSR: a weighted bincount over the nonzeros,
which sums each output entry left to right). Iterations follow the paper's
algorithms step by step, in the paper's order and notation:

  * ``cta``  -- Algorithm 1.1 with H = A Aᵀ (Sec. 3, Eqs. F_t, eqcoeff, CTAGEN7,
               CTAGEN7A) and the t-cycling of Sec. 5.1.
  * ``ta``   -- Algorithms 2.1, 2.2 and 2.5 (Sec. 4, Eqs. pivotTA, alph, vr,
               eqlem2, Cor. cor1), and the hybrid CTA -> TA of Sec. 5.2.

Where the paper is silent or ambiguous the oracle takes one documented reading;
each is named in the docstring of the function that implements it.

Parity pins: every function here is pinned by the tests in
``tests/test_oracle_*.py`` against closed forms, theorems and textbook
equivalences stated in the paper (nothing is pinned against the CUDA path).
"""
from .ops import Operator, NormalOperator, make_operator
from .cta import (schedule, hankel_solve, cta_chain, cta_step, cta_solve, CTAResult,
                  PINGPONG, SAWTOOTH, FIXED)
from .ta import ta_solve, ta_fixed_rho, ta_minnorm_bisect, ta_minnorm, TAResult, MinNormResult
from .status import Status, Reason

__all__ = [
    "Operator", "NormalOperator", "make_operator",
    "schedule", "hankel_solve", "cta_chain", "cta_step", "cta_solve", "CTAResult",
    "PINGPONG", "SAWTOOTH", "FIXED",
    "ta_solve", "ta_fixed_rho", "ta_minnorm_bisect", "ta_minnorm", "TAResult", "MinNormResult",
    "Status", "Reason",
]
