"""Pins for the oracle's direct solvers and problem definitions (CPU only).

x* = (A^T J A)^{-1} A^T J b (eq. (1.2)-(1.3)) is pinned by an exact rational
solve on small integer instances, by ordinary least squares when q = 0 (Sec. 1),
and the QR-Cholesky method (Sec. 1) and the normal-equation Cholesky solve are
pinned against each other on Gaussian instances.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


@pytest.mark.parametrize("seed,p,q,n", [(1, 6, 2, 2), (2, 7, 3, 3), (3, 9, 3, 4), (4, 5, 1, 4), (5, 8, 0, 3)])
def test_direct_solvers_match_exact_rationals(seed, p, q, n):
    for s in range(seed, seed + 40):
        inst = W.tiny_integer_instance(p, q, n, s)
        if O.is_spd(O.normal_matrix(inst.A, p)) and np.linalg.cond(O.normal_matrix(inst.A, p)) < 1e6:
            break
    else:
        pytest.skip("no SPD draw")
    exact = np.array([float(v) for v in O.exact_solve_fraction(inst.A, inst.b, p)])
    for fn in (O.qr_cholesky_solve, O.normal_equation_solve):
        x = fn(inst.A, inst.b, p)
        assert np.allclose(x, exact, rtol=1e-10, atol=1e-10), (fn.__name__, x, exact)


def test_q_zero_is_ordinary_least_squares():
    inst = W.dense_gaussian(60, 0, 9, 0.0, 11)
    x_ls = np.linalg.lstsq(inst.A, inst.b, rcond=None)[0]
    x = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    assert np.linalg.norm(x - x_ls) <= 1e-12 * np.linalg.norm(x_ls)


def test_qr_cholesky_agrees_with_normal_equations_config1():
    inst = W.config1()
    x1 = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x2 = O.normal_equation_solve(inst.A, inst.b, inst.p)
    assert np.linalg.norm(x1 - x2) <= 1e-13 * np.linalg.norm(x1)
    assert O.relres(inst.A, inst.b, inst.p, x1) < 1e-14


def test_split_identity_and_rhs():
    """A^T J A = A_1^T A_1 - A_2^T A_2 and A^T J b = A_1^T b_1 - A_2^T b_2 (Sec. 2), against explicit J."""
    inst = W.dense_gaussian(13, 5, 4, 0.5, 3)
    J = np.diag(np.r_[np.ones(13), -np.ones(5)])
    assert np.allclose(O.normal_matrix(inst.A, 13), inst.A.T @ J @ inst.A, atol=1e-12)
    assert np.allclose(O.rhs_bar(inst.A, inst.b, 13), inst.A.T @ J @ inst.b, atol=1e-12)
    x = np.arange(4.0)
    assert np.allclose(O.residual(inst.A, inst.b, 13, x), inst.A.T @ J @ (inst.b - inst.A @ x), atol=1e-12)


def test_solution_minimises_indefinite_form():
    """x* is the unique minimiser of (b-Ax)^T J (b-Ax) (eq. (1.1)); perturbations raise it."""
    inst = W.config1()
    J = np.r_[np.ones(inst.p), -np.ones(inst.q)]
    f = lambda x: float(((inst.b - inst.A @ x) ** 2 * J).sum())
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    rng = np.random.default_rng(0)
    for _ in range(20):
        d = rng.standard_normal(inst.n) * 1e-3
        assert f(xs + d) > f(xs)


def test_spd_detection_and_theorem21_radius():
    """Theorem 2.1: rho(Abar1^{-1} Abar2) < 1 whenever (1.3) holds; and fails when A_2 dominates."""
    inst = W.config1()
    rho = O.sp_spectral_radius(inst.A, inst.p)
    assert 0.0 <= rho < 1.0
    bad = W.dense_gaussian(60, 40, 10, 3.0, 2)
    assert not O.is_spd(O.normal_matrix(bad.A, bad.p))
