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
