"""GPU parity of SP-RK-RGS (Alg. 2) and SP-SCD (Alg. 5) against the CPU oracle.

Both sides draw from Philox4x32-10 with the same (seed, chain, k, t) counters, so
short inner runs follow the same index sequence and agree to rounding; full solves
converge to the unique x* (Theorems 3.2 and 4.1), checked to 1e-10.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import colmajor, relerr, to_np_colmajor, vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ils():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2203_15340_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def c1():
    inst = W.config1()
    return inst, O.qr_cholesky_solve(inst.A, inst.b, inst.p)


def run(ils, inst, method, tol=1e-12, **opt):
    import torch
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(method=method, **opt))
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=tol, allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    s.close()
    return out, info


@pytest.mark.parametrize("sampler", [0, 1])
def test_scd_config1_converges(ils, c1, sampler):
    inst, xs = c1
    x, info = run(ils, inst, ils.ILS_SP_SCD, scd_sampler=sampler)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
    _, oinfo = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=1e-12,
                              sampler="rank" if sampler == 0 else "greedy")
    assert abs(info.outer_iters - oinfo.outer_iters) <= 2
    assert 0.5 * sum(oinfo.inner_iters) <= info.inner_iters <= 2.0 * sum(oinfo.inner_iters)


@pytest.mark.parametrize("sampler", [0, 1])
def test_scd_trajectory_matches_oracle(ils, c1, sampler):
    """One outer iteration with a fixed number of inner steps follows the oracle's picks."""
    inst, _ = c1
    steps = 120
    x, info = run(ils, inst, ils.ILS_SP_SCD, tol=0.0, max_outer=1, max_inner=steps, theta=1e-300,
                  scd_sampler=sampler, seed=77)
    xo, oinfo = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps, theta=1e-300,
                               sampler="rank" if sampler == 0 else "greedy", seed=77)
    assert info.inner_iters == steps == oinfo.inner_iters[0]
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)


def test_rk_rgs_config1_converges(ils, c1):
    inst, xs = c1
    x, info = run(ils, inst, ils.ILS_SP_RK_RGS, seed=3)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
    _, oinfo = O.sp_rk_rgs_solve(inst.A, inst.b, inst.p, tol=1e-12, seed=3)
    assert abs(info.outer_iters - oinfo.outer_iters) <= 2


def test_rk_rgs_trajectory_matches_oracle(ils, c1):
    inst, _ = c1
    steps = 300
    x, info = run(ils, inst, ils.ILS_SP_RK_RGS, tol=0.0, max_outer=1, max_inner=steps, check_every=10 ** 9,
                  seed=5)
    xo, oinfo = O.sp_rk_rgs_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps,
                                  check_every=10 ** 9, seed=5)
    assert info.inner_iters == steps
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


def test_rk_rgs_same_index_is_coordinate_descent(ils, c1):
    """j2 = j1 (SP-RCD, Sec. 4) also converges to x*."""
    inst, xs = c1
    x, info = run(ils, inst, ils.ILS_SP_RK_RGS, scd_sampler=2, seed=9)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10


def test_rk_rgs_tall_block_in_global_scratch(ils):
    """p too large for shared memory: w and e stream through the global scratch slice."""
    inst = W.dense_gaussian(30000, 3000, 24, 0.3, 31)
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = run(ils, inst, ils.ILS_SP_RK_RGS, seed=1)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10


def test_randomized_many_rhs(ils):
    import torch
    inst = W.dense_gaussian(300, 60, 20, 0.3, 41, k=3)
    Xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    for method in (ils.ILS_SP_SCD, ils.ILS_SP_RK_RGS):
        s = ils.Solver(colmajor(inst.A), inst.p, ils.options(method=method, seed=2))
        X = torch.zeros((3, 20), dtype=torch.float64, device="cuda")
        info = s.solve_many(colmajor(inst.b), X, tol=1e-12)
        Xg = to_np_colmajor(X)
        for j in range(3):
            assert relerr(Xg[:, j], Xs[:, j]) <= 1e-10
        s.close()


# ---------------------------------------------------------------------------------------
# Pick sequences, fixed alpha, the Gram-space RK-RGS, the warm inner start, the alias draws
# ---------------------------------------------------------------------------------------

def gpu_picks(ils, inst, method, steps, per_step=1, **opt):
    """Run one outer iteration of `steps` inner steps and return the recorded picks and x."""
    import torch
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(method=method, **opt))
    picks = torch.full((steps * per_step,), -1, dtype=torch.int32, device="cuda")
    s.record_picks(picks)
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=0.0, allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    torch.cuda.synchronize()
    out = picks.cpu().numpy(), x.cpu().numpy(), info
    s.close()
    return out


@pytest.mark.parametrize("sampler,alpha", [("greedy", None), ("rank", None), ("fixed_rank", 1), ("fixed_rank", 2),
                                           ("fixed_rank", 17), ("fixed_rank", 50)])
def test_scd_pick_sequence_matches_oracle(ils, c1, sampler, alpha):
    """The chain picks exactly the oracle's indices (tie-free |r|): alpha = n is the greedy
    Motzkin rule (Sec. 4), the rank sampler is Alg. 5's law, fixed alpha its Sec. 4 variant."""
    inst, _ = c1
    steps = 120
    opt = dict(max_outer=1, max_inner=steps, theta=1e-300, seed=77)
    if sampler == "greedy":
        opt["scd_sampler"] = 1
    elif sampler == "fixed_rank":
        opt.update(alpha_mode=1, alpha_fixed=alpha)
    picks, x, info = gpu_picks(ils, inst, ils.ILS_SP_SCD, steps, **opt)
    xo, oinfo = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps, theta=1e-300,
                               sampler=sampler, alpha=alpha, seed=77, record=True)
    assert list(picks) == oinfo.picks
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)


def test_scd_greedy_through_alpha_n(ils, c1):
    inst, _ = c1
    kw = dict(max_outer=1, max_inner=60, theta=1e-300)
    p1, _, _ = gpu_picks(ils, inst, ils.ILS_SP_SCD, 60, scd_sampler=1, **kw)
    p2, _, _ = gpu_picks(ils, inst, ils.ILS_SP_SCD, 60, alpha_mode=1, alpha_fixed=inst.n, **kw)
    assert np.array_equal(p1, p2)


@pytest.mark.parametrize("n", [1500, 3000, 5000, 9000])
def test_scd_register_layouts_follow_oracle(ils, n):
    """Every register layout of the SCD chain (1, 2, 4 entries per thread of 1024; 16 and 32
    of 512) follows the oracle's picks, including the radix path for ranks above 8."""
    inst = W.dense_gaussian(n + 3000, 100, n, 0.02, 60 + n)
    steps = 80
    picks, x, _ = gpu_picks(ils, inst, ils.ILS_SP_SCD, steps, max_outer=1, max_inner=steps, theta=1e-300, seed=5)
    xo, oinfo = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps, theta=1e-300,
                               seed=5, record=True)
    assert list(picks) == oinfo.picks
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo)


def test_rk_rgs_draws_match_oracle(ils, c1):
    inst, _ = c1
    steps = 200
    picks, x, _ = gpu_picks(ils, inst, ils.ILS_SP_RK_RGS, steps, per_step=2, max_outer=1, max_inner=steps,
                            check_every=10 ** 9, seed=5)
    xo, oinfo = O.sp_rk_rgs_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps,
                                  check_every=10 ** 9, seed=5, record=True)
    assert [tuple(p) for p in picks.reshape(-1, 2)] == oinfo.picks
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("n", [50, 700, 3000])
def test_rk_rgs_gram_form_follows_oracle(ils, n):
    """The Gram-space chain follows the oracle's Gram form (and so the column form) step by step."""
    inst = W.config1() if n == 50 else W.dense_gaussian(n + 600, 200, n, 0.2, 70 + n)
    steps = 300
    _, x, info = gpu_picks(ils, inst, ils.ILS_SP_RK_RGS, steps, per_step=2, max_outer=1, max_inner=steps,
                           check_every=10 ** 9, seed=6, inner_form=1)
    xo, _ = O.sp_rk_rgs_gram_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps,
                                   check_every=10 ** 9, seed=6)
    assert info.inner_iters == steps
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("method,form", [(2, 0), (1, 0), (1, 1)])
def test_warm_inner_start_converges_and_follows_oracle(ils, c1, method, form):
    """z = x_k / beta = x_k starts (correction form on the device): a full solve reaches x*
    with fewer inner steps than the cold start, and short runs follow the oracle's warm form."""
    inst, xs = c1
    opt = dict(seed=3, inner_form=form) if method == 1 else dict(seed=3)
    x, info = run(ils, inst, method, warm_inner=1, **opt)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
    _, cold = run(ils, inst, method, **opt)
    assert info.inner_iters < cold.inner_iters
    fn = {2: O.sp_scd_solve, 1: O.sp_rk_rgs_gram_solve if form else O.sp_rk_rgs_solve}[method]
    kw = dict(max_outer=3, max_inner=150, seed=8)
    if method == 1:
        kw["check_every"] = 10 ** 9
    else:
        kw["theta"] = 1e-300
    xo, _ = fn(inst.A, inst.b, inst.p, tol=0.0, warm_inner=True, **kw)
    xg, _ = run(ils, inst, method, tol=0.0, warm_inner=1, inner_form=form if method == 1 else 0, **kw)
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)


def test_alias_sampler_law_and_convergence(ils, c1):
    """Alias draws follow ||A_1(:,j)||^2 / ||A_1||_F^2 (chi-square over 60000 draws) and the
    solve converges to x*."""
    from scipy import stats
    inst, xs = c1
    steps = 30000
    picks, _, _ = gpu_picks(ils, inst, ils.ILS_SP_RK_RGS, steps, per_step=2, max_outer=1, max_inner=steps,
                            check_every=10 ** 9, seed=12, sampler=1)
    norms2 = np.einsum("ij,ij->j", inst.A[: inst.p], inst.A[: inst.p])
    expected = norms2 / norms2.sum() * picks.size
    counts = np.bincount(picks, minlength=inst.n)
    assert picks.min() >= 0 and stats.chisquare(counts, expected).pvalue > 1e-4
    x, info = run(ils, inst, ils.ILS_SP_RK_RGS, sampler=1, seed=4)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10


@pytest.mark.parametrize("method", [1, 2])
def test_theta_schedule_follows_oracle(ils, c1, method):
    """theta_k = max(theta gamma^k, theta_min): four outer iterations follow the oracle's
    schedule (the same inner counts, the same x to rounding; SCD by its greedy rule, RK-RGS by
    the shared Philox draws), and a full solve with the schedule reaches x*."""
    inst, xs = c1
    sched = dict(theta_decay=0.5, theta_min=1e-6)
    if method == 2:
        xg, ig = run(ils, inst, method, tol=0.0, max_outer=4, scd_sampler=1, **sched)
        xo, io = O.sp_scd_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=4, sampler="greedy", **sched)
    else:
        xg, ig = run(ils, inst, method, tol=0.0, max_outer=4, seed=4, check_every=25, **sched)
        xo, io = O.sp_rk_rgs_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=4, seed=4, check_every=25, **sched)
    assert ig.inner_iters == sum(io.inner_iters)
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    x, info = run(ils, inst, method, seed=6, **sched)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
