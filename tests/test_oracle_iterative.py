"""Pins for the oracle's SP, SP-RK-RGS and SP-SCD methods (CPU only).

Each check comes from a statement of the paper that does not restate the
oracle's own formula: Theorem 2.1 (energy-norm contraction by rho, obtained
here from a generalized eigenvalue solve), Theorem 3.1 (the inner fixed point of
RK-RGS is the SP iterate), the Pythagorean step of Theorem 3.2's proof, the
reduction of RK-RGS with j1 = j2 to coordinate descent (Sec. 4), the exact energy
decrease of Theorem 4.1's proof, the alpha = n (Motzkin) special case, and the
iteration counts printed in Tables 2-3.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


@pytest.fixture(scope="module")
def c1():
    inst = W.config1()
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    return inst, xs


def relerr(x, xs):
    return np.linalg.norm(x - xs) / np.linalg.norm(xs)


def test_sp_converges_to_direct_solution(c1):
    inst, xs = c1
    x, info = O.sp_solve(inst.A, inst.b, inst.p, tol=1e-12)
    assert info.converged and relerr(x, xs) <= 1e-10
    assert 3 <= info.outer_iters <= 20


def test_sp_energy_contraction_theorem21(c1):
    """||x_{k+1} - x*||_{Abar1} <= rho ||x_k - x*||_{Abar1}; the ratio tends to rho."""
    inst, xs = c1
    A1 = inst.A[: inst.p]
    G1 = A1.T @ A1
    rho = O.sp_spectral_radius(inst.A, inst.p)
    x0 = np.random.default_rng(1).standard_normal(inst.n)
    _, info = O.sp_solve(inst.A, inst.b, inst.p, x0=x0, tol=1e-14, max_outer=6, record=True)
    errs = [O.energy_norm(x - xs, G1) for x in info.iterates]
    ratios = [errs[k + 1] / errs[k] for k in range(len(errs) - 1)]
    assert all(r <= rho * (1 + 1e-6) for r in ratios), (ratios, rho)
    assert ratios[-1] >= 0.5 * rho  # the bound is attained asymptotically


def test_sp_q_zero_one_step():
    """q = 0: B = 0, so one SP step gives the least-squares solution (Sec. 1)."""
    inst = W.dense_gaussian(80, 0, 12, 0.0, 4)
    x, info = O.sp_solve(inst.A, inst.b, inst.p, tol=1e-13)
    x_ls = np.linalg.lstsq(inst.A, inst.b, rcond=None)[0]
    assert info.outer_iters == 1 and relerr(x, x_ls) < 1e-12


def test_sp_multi_rhs_columns_independent():
    inst = W.dense_gaussian(90, 20, 10, 0.3, 8, k=3)
    X, info = O.sp_solve(inst.A, inst.b, inst.p, tol=1e-12)
    for j in range(3):
        xj, _ = O.sp_solve(inst.A, inst.b[:, j], inst.p, tol=1e-12)
        assert np.allclose(X[:, j], xj, rtol=0, atol=1e-12 * np.linalg.norm(xj))


def test_paper_table_iteration_counts():
    """Tables 2-3 print SP IT = 1 at RR < 1e-6 from x0 = 0 on the rand / 7*eye workload.

    Replayed at p = 4000, n = q = 1300 (the p/n ratio of Table 3's first column).
    lambda_min(Abar1) grows like p while the 7*eye block does not, so the replay
    scales the diagonal to keep rho(Abar1^{-1} Abar2) at the paper-size value
    (about 0.17 for p = 30000, n = 13000).
    """
    gold = json.load(open(GOLD))
    assert all(v == 1 for row in gold["printed"] for v in row["SP_IT"])
    p, n = 4000, 1300
    lam = lambda pp, nn: pp / 12.0 * (1.0 - math.sqrt(nn / pp)) ** 2  # U[0,1) Marchenko-Pastur edge
    diag = 7.0 * math.sqrt(lam(p, n) / lam(30000, 13000))
    inst = W.paper_table_workload(p, n, n, seed=0, diag=diag)
    assert O.is_spd(O.normal_matrix(inst.A, p))
    assert abs(O.sp_spectral_radius(inst.A, p) - 49.0 / lam(30000, 13000)) < 0.02
    tol = math.sqrt(gold["stop_rr"])
    x, info = O.sp_solve(inst.A, inst.b, p, tol=tol, max_outer=gold["max_outer"])
    assert info.outer_iters == 1
    assert O.paper_rr(inst.A, inst.b, p, x) < gold["stop_rr"]
    # SP-SCD: the printed IT is between 1 and 2 on average (Tables 2-5).
    _, info2 = O.sp_scd_solve(inst.A, inst.b, p, tol=tol, max_outer=3, max_inner=5 * n, theta=1e-3)
    assert 1 <= info2.outer_iters <= 2 and info2.converged


def test_rk_rgs_inner_fixed_point_theorem31(c1):
    """With a tight inner solve the outer iterates of SP-RK-RGS equal SP's (Theorem 3.1)."""
    inst, xs = c1
    small = W.dense_gaussian(60, 15, 6, 0.2, 21)
    _, sp = O.sp_solve(small.A, small.b, small.p, tol=1e-30, max_outer=3, record=True)
    _, rk = O.sp_rk_rgs_solve(small.A, small.b, small.p, tol=1e-30, max_outer=3, theta=1e-9,
                              max_inner=200000, check_every=6, record=True)
    for a, b in zip(sp.iterates, rk.iterates):
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(sp.iterates[-1])


def test_rgs_pythagorean_step_theorem32():
    """With w = w* = A_1 z*, an RGS step satisfies
    ||A_1(z~ - z*)||^2 = ||A_1(z - z*)||^2 - ||A_1(z~ - z)||^2 (proof of Theorem 3.2)."""
    rng = np.random.default_rng(3)
    A1 = rng.standard_normal((25, 7))
    norms2, _ = O.column_cumsum(A1)
    zs = rng.standard_normal(7)
    ws = A1 @ zs
    z = rng.standard_normal(7)
    for j in range(7):
        zt = O.rgs_step(A1, z, ws, j, norms2)
        lhs = np.sum((A1 @ (zt - zs)) ** 2)
        rhs = np.sum((A1 @ (z - zs)) ** 2) - np.sum((A1 @ (zt - z)) ** 2)
        assert abs(lhs - rhs) <= 1e-10 * np.sum((A1 @ (z - zs)) ** 2)
        # orthogonality of A_1(z~ - z*) to column j
        assert abs(A1[:, j] @ (A1 @ (zt - zs))) <= 1e-10 * np.linalg.norm(A1[:, j]) * np.linalg.norm(A1 @ (z - zs))


def test_rk_projection_satisfies_row():
    """After the RK step, the chosen equation A_1(:,j)^T w = bhat_j holds exactly (Sec. 3.1)."""
    rng = np.random.default_rng(4)
    A1 = rng.standard_normal((20, 5))
    norms2, _ = O.column_cumsum(A1)
    w = rng.standard_normal(20)
    bhat = rng.standard_normal(5)
    for j in range(5):
        w2 = O.rk_step(A1, w, bhat, j, norms2)
        assert abs(A1[:, j] @ w2 - bhat[j]) < 1e-12 * (1 + abs(bhat[j]))
        d = w2 - w  # the change is along column j
        assert np.linalg.matrix_rank(np.c_[d, A1[:, j]], tol=1e-10) == 1


def test_rk_rgs_same_index_is_coordinate_descent():
    """j1 = j2 = j turns the RK-RGS step into z_j += (bhat_j - Abar1(j,:) z) / Abar1_jj (Sec. 4)."""
    rng = np.random.default_rng(6)
    A1 = rng.standard_normal((30, 6))
    G1 = A1.T @ A1
    norms2, _ = O.column_cumsum(A1)
    bhat = rng.standard_normal(6)
    w = np.zeros(30)
    z = np.zeros(6)
    for t in range(40):
        j = int(rng.integers(6))
        w = O.rk_step(A1, w, bhat, j, norms2)
        z_new = O.rgs_step(A1, z, w, j, norms2)
        cd = z.copy()
        cd[j] += (bhat[j] - G1[j] @ z) / G1[j, j]
        assert np.allclose(z_new, cd, atol=1e-12 * (1 + np.abs(cd).max()))
        z = z_new


def test_scd_energy_decrease_theorem41():
    """||beta_t - beta*||^2_{Abar1} = ||beta_{t-1} - beta*||^2_{Abar1} - r_j^2 / Abar1_jj, exactly."""
    rng = np.random.default_rng(7)
    A1 = rng.standard_normal((40, 8))
    G1 = A1.T @ A1
    bhat = rng.standard_normal(8)
    bs = np.linalg.solve(G1, bhat)
    beta = np.zeros(8)
    r = bhat.copy()
    e = lambda v: float((v - bs) @ G1 @ (v - bs))
    for t in range(30):
        j = int(rng.integers(8))
        rj = r[j]
        before = e(beta)
        beta, r = O.scd_step(G1, beta, r, j)
        assert abs(e(beta) - (before - rj * rj / G1[j, j])) <= 1e-9 * before
        assert np.allclose(r, bhat - G1 @ beta, atol=1e-10)


def test_scd_rank_law_equals_literal_law():
    """The rank sampler has exactly the law of alpha ~ U{1..n} + uniform alpha-subset + argmax."""
    rng = np.random.default_rng(8)
    for n in range(1, 8):
        absr = rng.permutation(n) + rng.random(n) * 0.1 + 0.5
        assert np.allclose(O.scd_rank_law(absr), O.scd_literal_law(absr), atol=1e-14)


def test_scd_rank_sampler_inverse_cdf():
    n = 9
    probs = np.array([(n + 1) / (n * i * (i + 1)) for i in range(1, n + 1)])
    assert abs(probs.sum() - 1) < 1e-14
    counts = np.zeros(n)
    rng = np.random.default_rng(9)
    for u in rng.random(20000):
        counts[O.scd_rank_from_uniform(u, n) - 1] += 1
    assert stats.chisquare(counts, 20000 * probs).pvalue > 1e-3
    assert O.scd_rank_from_uniform(0.0, n) == 1
    assert O.scd_rank_from_uniform(1.0 - 1e-16, n) == n


def test_scd_literal_sampler_empirical_law():
    rng = np.random.default_rng(10)
    r = np.array([0.3, -2.0, 1.1, 0.05, -0.7])
    counts = np.zeros(5)
    for _ in range(20000):
        a = int(rng.integers(1, 6))
        counts[O.scd_pick_literal(r, a, rng.choice(5, size=a, replace=False))] += 1
    expect = 20000 * O.scd_literal_law(np.abs(r))
    assert stats.chisquare(counts, expect).pvalue > 1e-3


def test_scd_greedy_is_argmax():
    r = np.array([0.5, -3.0, 3.0, 1.0])
    assert O.scd_pick_literal(r, 4, range(4)) == 1  # tie |r|=3: lowest index


@pytest.mark.parametrize("sampler", ["rank", "literal", "greedy"])
def test_scd_converges(c1, sampler):
    inst, xs = c1
    x, info = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=1e-12, sampler=sampler)
    assert info.converged and relerr(x, xs) <= 1e-10


def test_rk_rgs_converges(c1):
    inst, xs = c1
    x, info = O.sp_rk_rgs_solve(inst.A, inst.b, inst.p, tol=1e-12)
    assert info.converged and relerr(x, xs) <= 1e-10


# ---------------------------------------------------------------------------------------
# Fixed subset size alpha (Sec. 4: alpha = n is the Motzkin greedy rule), the error
# certificate, the inner warm start and the Gram-space form of RK-RGS.
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 5, 7])
def test_scd_fixed_rank_law_equals_literal_law(n):
    """argmax over a uniform alpha-subset, enumerated subset by subset, has the rank law
    C(n-i, alpha-1) / C(n, alpha) for every alpha (tie-free |r|)."""
    absr = np.random.default_rng(n).permutation(np.arange(1, n + 1)).astype(float)
    for alpha in range(1, n + 1):
        lit = O.scd_fixed_literal_law(absr, alpha)
        assert np.allclose(lit, O.scd_fixed_rank_law(absr, alpha), rtol=0, atol=1e-15), alpha
        assert abs(lit.sum() - 1.0) <= 1e-14


@pytest.mark.parametrize("n,alpha", [(7, 1), (7, 3), (50, 1), (50, 2), (50, 16), (50, 17), (50, 40), (50, 50),
                                     (301, 5), (301, 120)])
def test_scd_fixed_rank_inverse_cdf(n, alpha):
    """On a fine uniform grid of u the sampled rank has the law C(n-i, alpha-1)/C(n, alpha):
    both the bisection form (alpha <= 16) and the scan form (alpha > 16)."""
    us = (np.arange(100000) + 0.5) / 100000
    ranks = np.array([O.scd_fixed_rank_from_uniform(u, n, alpha) for u in us])
    assert ranks.min() >= 1 and ranks.max() <= n - alpha + 1
    freq = np.bincount(ranks, minlength=n + 1)[1:] / us.size
    law = np.array([math.comb(n - i, alpha - 1) / math.comb(n, alpha) for i in range(1, n + 1)])
    assert np.max(np.abs(freq - law)) <= 2e-5


def test_scd_fixed_alpha_n_is_greedy(c1):
    """alpha = n: the subset is everything, so the fixed-alpha sampler makes the greedy picks."""
    inst, _ = c1
    kw = dict(tol=0.0, max_outer=1, max_inner=80, theta=1e-300, record=True)
    _, a = O.sp_scd_solve(inst.A, inst.b, inst.p, sampler="fixed_rank", alpha=inst.n, **kw)
    _, g = O.sp_scd_solve(inst.A, inst.b, inst.p, sampler="greedy", **kw)
    assert a.picks == g.picks and len(a.picks) == 80


@pytest.mark.parametrize("alpha", [1, 2, 17])
def test_scd_fixed_alpha_converges(c1, alpha):
    inst, xs = c1
    x, info = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=1e-12, sampler="fixed_rank", alpha=alpha, seed=4)
    assert info.converged and np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_error_certificate_bounds_the_error():
    """kappa(H) relres bounds ||x - x*|| / ||x*|| for any x (checked on perturbed iterates
    of three instances), and kappa of a diagonal H is the ratio of its extreme entries."""
    rng = np.random.default_rng(9)
    for seed in range(3):
        inst = W.dense_gaussian(120, 30, 12, 0.3, 50 + seed)
        xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
        kap = O.normal_matrix_condition(inst.A, inst.p)
        for scale in (1e-2, 1e-6, 1e-11):
            x = xs + scale * np.linalg.norm(xs) * rng.standard_normal(xs.shape) / math.sqrt(xs.size)
            err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
            assert err <= O.error_certificate(inst.A, inst.b, inst.p, x, kappa=kap) * (1 + 1e-6)
    d1, d2 = np.array([4.0, 3.0, 5.0]), np.array([1.0, 2.0, 0.5])
    A = np.vstack([np.diag(d1), np.diag(d2)])
    lam = d1 ** 2 - d2 ** 2
    assert abs(O.normal_matrix_condition(A, 3) - lam.max() / lam.min()) <= 1e-13 * lam.max() / lam.min()


def test_rk_rgs_gram_form_equals_column_form(c1):
    """Gram-space RK-RGS follows the column form step for step under the same draws."""
    inst, _ = c1
    kw = dict(tol=0.0, max_outer=2, max_inner=300, check_every=10 ** 9, seed=5)
    for same in (False, True):
        xc, _ = O.sp_rk_rgs_solve(inst.A, inst.b, inst.p, same_index=same, **kw)
        xg, _ = O.sp_rk_rgs_gram_solve(inst.A, inst.b, inst.p, same_index=same, **kw)
        assert np.linalg.norm(xg - xc) <= 1e-12 * np.linalg.norm(xc)


@pytest.mark.parametrize("solver", ["rk_rgs", "rk_rgs_gram", "scd"])
def test_warm_inner_start_keeps_the_sp_step(c1, solver):
    """With the inner solve run to convergence, one outer step equals SP's step from either
    start (the inner fixed point is Abar1^{-1} bhat, Theorem 3.1), and a full warm-started
    solve converges to x* with fewer inner steps than the cold one."""
    inst, xs = c1
    fn = {"rk_rgs": O.sp_rk_rgs_solve, "rk_rgs_gram": O.sp_rk_rgs_gram_solve, "scd": O.sp_scd_solve}[solver]
    x0 = xs + 0.1 * np.random.default_rng(1).standard_normal(inst.n)
    x_sp, _ = O.sp_solve(inst.A, inst.b, inst.p, x0=x0, tol=0.0, max_outer=1)
    x_w, _ = fn(inst.A, inst.b, inst.p, x0=x0, tol=0.0, max_outer=1, theta=1e-13, max_inner=400000, warm_inner=True)
    assert np.linalg.norm(x_w - x_sp) <= 1e-10 * np.linalg.norm(x_sp)
    _, cold = fn(inst.A, inst.b, inst.p, tol=1e-12, seed=3)
    xw, warm = fn(inst.A, inst.b, inst.p, tol=1e-12, seed=3, warm_inner=True)
    assert warm.converged and np.linalg.norm(xw - xs) <= 1e-10 * np.linalg.norm(xs)
    assert sum(warm.inner_iters) < sum(cold.inner_iters)


def test_theta_schedule_closed_form():
    """theta_k = max(theta gamma^k, theta_min); gamma = 1 or <= 0 keeps theta."""
    assert O.theta_at(0.1, 0, 0.5) == 0.1
    assert abs(O.theta_at(0.1, 3, 0.5) - 0.0125) < 1e-18
    assert O.theta_at(0.1, 10, 0.5, theta_min=1e-3) == 1e-3
    assert O.theta_at(0.1, 7, 1.0) == 0.1 and O.theta_at(0.1, 7, 0.0) == 0.1


@pytest.mark.parametrize("solver", ["rk_rgs", "scd"])
def test_theta_schedule_constant_reproduces(c1, solver):
    """A schedule with gamma = 1 is the constant inner stop: the same iterates and counts."""
    inst, _ = c1
    fn = O.sp_rk_rgs_solve if solver == "rk_rgs" else O.sp_scd_solve
    x0, i0 = fn(inst.A, inst.b, inst.p, tol=1e-10, max_outer=60, seed=3)
    x1, i1 = fn(inst.A, inst.b, inst.p, tol=1e-10, max_outer=60, seed=3, theta_decay=1.0, theta_min=0.5)
    assert np.array_equal(x0, x1) and i0.inner_iters == i1.inner_iters


def test_theta_schedule_bounds_each_outer_step(c1):
    """Where an inner solve stopped on its test, z solves Abar1 z = bhat to theta_k ||r_k||,
    so x_{k+1} lies within ||Abar1^{-1}|| theta_k ||r_k|| of the exact SP step
    Abar1^{-1}(Abar2 x_k + bbar): the schedule's theta_k (not theta) is what bounds it."""
    inst, _ = c1
    G1, G2 = O.gram_blocks(inst.A, inst.p)
    bb = O.rhs_bar(inst.A, inst.b, inst.p)
    inv_norm = 1.0 / np.linalg.eigvalsh(G1)[0]
    gamma, tmin = 0.3, 1e-6
    x, info = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=1e-11, max_outer=40, seed=5, record=True,
                             theta_decay=gamma, theta_min=tmin)
    it = info.iterates
    checked = 0
    for k in range(len(it) - 1):
        if info.inner_iters[k] >= 200 * inst.n:
            continue
        r = O.residual(inst.A, inst.b, inst.p, it[k])
        sp = np.linalg.solve(G1, G2 @ it[k] + bb)
        bound = inv_norm * O.theta_at(0.1, k, gamma, tmin) * np.linalg.norm(r)
        assert np.linalg.norm(it[k + 1] - sp) <= bound * (1 + 1e-9) + 1e-13
        checked += 1
    assert checked >= 3 and info.converged
