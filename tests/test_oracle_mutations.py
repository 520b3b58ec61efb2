"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case patches one plausible slip into the oracle (a shifted moment index,
a flipped sign, a transposed operand, the paper's own "(1+alpha)" typo, the
wrong t-cycle, ...) and asserts that at least one pin in
test_oracle_pins.py fails on it. The mistakes live only inside these tests.
"""
import numpy as np
import pytest

import oracle
import oracle.cta as ocx
import oracle.ops as oops
import oracle.ta as otx
import tests.test_oracle_pins as pins


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_mutation_shifted_moment_index(monkeypatch):
    orig = ocx.hankel_solve

    def bad(phi, t, pivot_tol=1e-12):
        shifted = [0.0] + list(phi[2:]) + [phi[-1]]
        return orig(shifted, t, pivot_tol)
    monkeypatch.setattr(ocx, "hankel_solve", bad)
    _fails(pins.test_Ft_is_the_least_squares_step, 2)


def test_mutation_residual_sign(monkeypatch):
    def bad_step(A, x, r, t, pivot_tol=1e-12):
        z, u, phi = ocx.cta_chain(A, r, t)
        alpha, rank = ocx.hankel_solve(phi, t, pivot_tol)
        x2, r2 = x.copy(), r.copy()
        for i in range(t):
            x2 += alpha[i] * z[i]
            r2 += alpha[i] * u[i]
        return x2, r2, alpha, rank, phi
    monkeypatch.setattr(ocx, "cta_step", bad_step)
    monkeypatch.setattr(oracle, "cta_step", bad_step)
    _fails(pins.test_Ft_is_the_least_squares_step, 1)


def test_mutation_x_update_uses_wrong_chain_vector(monkeypatch):
    def bad_chain(A, r, t):
        z, u, phi = ocx.__dict__["_orig_chain"](A, r, t)
        return [A.rmatvec(ui) for ui in u], u, phi      # A^T H^i r instead of A^T H^{i-1} r
    monkeypatch.setitem(ocx.__dict__, "_orig_chain", ocx.cta_chain)
    monkeypatch.setattr(ocx, "cta_chain", bad_chain)
    _fails(pins.test_Ft_equals_t_lsqr_steps, 2)


def test_mutation_transposed_operand(monkeypatch):
    monkeypatch.setattr(oops.Operator, "rmatvec",
                        lambda self, r: np.bincount(self.row_of, weights=self.vals * r[self.colidx],
                                                    minlength=self.m)
                        if self.fmt == "csr" else self.A @ r)
    _fails(pins.test_csr_products_are_the_definition)


def test_mutation_paper_typo_one_plus_alpha(monkeypatch):
    """Sec. 3.4's remark prints (1+alpha); the TA update must use (1-alpha)."""
    import inspect
    src = inspect.getsource(otx._ta_loop)
    src = src.replace("bp = (1.0 - alpha) * bp", "bp = (1.0 + alpha) * bp")
    src = src.replace("x = (1.0 - alpha) * x", "x = (1.0 + alpha) * x")
    ns = dict(otx.__dict__)
    exec(compile(src, "<mutant>", "exec"), ns)
    monkeypatch.setattr(otx, "_ta_loop", ns["_ta_loop"])
    _fails(pins.test_ta_invariants_each_iteration)


def test_mutation_rho_growth_min(monkeypatch):
    """Alg. 2.2 grows rho with max{2 rho, (b-b')ᵀb/||c||}; min would stall at 0."""
    import inspect
    src = inspect.getsource(otx._ta_loop).replace("rho = max(2.0 * rho, db / cn)",
                                                  "rho = min(2.0 * rho, db / cn)")
    ns = dict(otx.__dict__)
    exec(compile(src, "<mutant>", "exec"), ns)
    monkeypatch.setattr(otx, "_ta_loop", ns["_ta_loop"])
    _fails(pins.test_ta_identity_golden)


def test_mutation_sawtooth_instead_of_pingpong(monkeypatch):
    monkeypatch.setattr(oracle, "schedule", lambda k, t_max, cycle=0: 1 + k % t_max)
    _fails(pins.test_schedule_matches_sec51_cycling)


def test_mutation_hankel_rhs_off_by_one(monkeypatch):
    import inspect
    src = inspect.getsource(ocx.hankel_solve).replace("g = [s[i] * phi[i + 1] for i in range(rank)]",
                                                      "g = [s[i] * phi[i + 2] for i in range(rank)]")
    ns = dict(ocx.__dict__)
    exec(compile(src, "<mutant>", "exec"), ns)
    monkeypatch.setattr(ocx, "hankel_solve", ns["hankel_solve"])
    monkeypatch.setattr(oracle, "hankel_solve", ns["hankel_solve"])
    _fails(pins.test_hankel_golden_closed_forms)


def test_mutation_lp_uses_c_instead_of_c_plus(monkeypatch):
    """Sec. 6: the LP form must replace c by c_+; keeping c breaks x' >= 0 and the golden."""
    import inspect
    src = inspect.getsource(otx._ta_loop).replace("c = np.maximum(c, 0.0)", "c = c")
    ns = dict(otx.__dict__)
    exec(compile(src, "<mutant>", "exec"), ns)
    monkeypatch.setattr(otx, "_ta_loop", ns["_ta_loop"])
    _fails(pins.test_ta_lp_identity_golden)
