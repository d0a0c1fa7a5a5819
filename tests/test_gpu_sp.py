"""GPU parity of the FP64 SP path (Alg. 1) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import colmajor, gemm_bound, relerr, to_np_colmajor, vec

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


def solve_gpu(ils, inst, tol=1e-12, x0=None, **opt):
    import torch
    solver = ils.Solver(colmajor(inst.A), inst.p, ils.options(**opt))
    x = vec(np.zeros(inst.n) if x0 is None else x0)
    info = solver.solve(vec(inst.b), x, x0_zero=x0 is None, tol=tol,
                        allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    solver.close()
    return out, info


# Shapes that cover full 64-wide tiles, ragged tails, a single column and K not a multiple of 16.
SHAPES = [(400, 100, 50), (37, 5, 1), (70, 9, 2), (130, 31, 31), (300, 77, 33), (500, 120, 65),
          (1000, 250, 130), (3001, 499, 257)]


@pytest.mark.parametrize("p,q,n", SHAPES)
def test_gram_cholesky_and_B_parity(ils, p, q, n):
    import torch
    inst = W.dense_gaussian(p, q, n, 0.3 * min(1.0, (p ** 0.5 - n ** 0.5) / (q ** 0.5 + n ** 0.5 + 1e-9)),
                            1000 + n)
    assert O.is_spd(O.normal_matrix(inst.A, p))
    s = ils.Solver(colmajor(inst.A), p, ils.options(route=ils.ILS_ROUTE_EXPLICIT))
    G1o, G2o = O.gram_blocks(inst.A, p)
    A1, A2 = inst.A[:p], inst.A[p:]
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    s.get_matrix(ils.MAT_GRAM1, out)
    G1 = to_np_colmajor(out)
    assert np.all(np.abs(G1 - G1o) <= gemm_bound(A1, A1) + 1e-300)
    assert np.array_equal(G1, G1.T)
    s.get_matrix(ils.MAT_GRAM2, out)
    G2 = to_np_colmajor(out)
    assert np.all(np.abs(G2 - G2o) <= gemm_bound(A2, A2) + 1e-300)
    s.get_matrix(ils.MAT_CHOL, out)
    L = to_np_colmajor(out)
    assert np.allclose(np.triu(L, 1), 0.0)
    # Backward error of the factor: ||L L^T - Abar1|| <= c n u ||Abar1||.
    assert np.linalg.norm(L @ L.T - G1o) <= 8 * n * 2.0 ** -53 * np.linalg.norm(G1o)
    s.get_matrix(ils.MAT_B, out)
    B = to_np_colmajor(out)
    Bo = np.linalg.solve(G1o, G2o)
    kappa = np.linalg.cond(G1o)
    assert np.linalg.norm(B - Bo) <= 64 * n * kappa * 2.0 ** -53 * max(np.linalg.norm(Bo), 1e-300) + 1e-14
    s.close()


def test_sp_config1_matches_oracle(ils):
    inst = W.config1()
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = solve_gpu(ils, inst, tol=1e-12)
    assert info.status == ils.ILS_OK
    assert relerr(x, xs) <= 1e-10
    _, oinfo = O.sp_solve(inst.A, inst.b, inst.p, tol=1e-12)
    assert abs(info.outer_iters - oinfo.outer_iters) <= 1
    assert info.relres <= 1e-12 and abs(info.relres - O.relres(inst.A, inst.b, inst.p, x)) <= 1e-13


def test_sp_trajectory_matches_oracle_iterates(ils):
    """x_k after max_outer = k updates equals the oracle's k-th SP iterate (Alg. 1 step 6)."""
    inst = W.config1()
    _, oinfo = O.sp_solve(inst.A, inst.b, inst.p, tol=0.0, max_outer=4, record=True)
    for k in range(0, 5):
        x, info = solve_gpu(ils, inst, tol=0.0, max_outer=k)
        assert info.outer_iters == k
        assert info.status == (ils.ILS_ERR_NO_CONVERGENCE if k < 5 else ils.ILS_OK)
        xo = oinfo.iterates[k]
        assert np.linalg.norm(x - xo) <= 1e-13 * max(np.linalg.norm(xo), 1.0)


def test_sp_warm_start_and_q_zero(ils):
    inst = W.config1()
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = solve_gpu(ils, inst, tol=1e-12, x0=xs + 1e-6)
    assert relerr(x, xs) <= 1e-10 and info.outer_iters <= 6
    ls = W.dense_gaussian(90, 0, 12, 0.0, 5)
    x, info = solve_gpu(ils, ls, tol=1e-13)
    assert info.outer_iters == 1
    assert relerr(x, np.linalg.lstsq(ls.A, ls.b, rcond=None)[0]) <= 1e-12


def test_sp_many_rhs(ils):
    import torch
    inst = W.dense_gaussian(700, 150, 60, 0.3, 12, k=11)  # two passes of up to 8 columns
    s = ils.Solver(colmajor(inst.A), inst.p)
    X = torch.zeros((11, 60), dtype=torch.float64, device="cuda")
    info = s.solve_many(colmajor(inst.b), X, tol=1e-12)
    Xg = to_np_colmajor(X)
    Xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    for j in range(11):
        assert relerr(Xg[:, j], Xs[:, j]) <= 1e-10
    assert info.relres <= 1e-12
    s.close()


def test_sp_config2_full_size(ils):
    inst = W.config2()
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = solve_gpu(ils, inst, tol=1e-12)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
    assert 5 <= info.outer_iters <= 12


def test_not_spd_and_nonfinite_inputs(ils):
    bad = W.dense_gaussian(60, 40, 10, 3.0, 2)  # A^T J A indefinite, A_1^T A_1 SPD
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(bad.A), bad.p)
    assert e.value.code == ils.ILS_ERR_NOT_SPD
    zc = W.dense_gaussian(60, 10, 6, 0.1, 3)
    zc.A[:, 2] = 0.0  # a zero column: A_1^T A_1 singular
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(zc.A), zc.p)
    assert e.value.code == ils.ILS_ERR_NOT_SPD
    nan = W.dense_gaussian(60, 10, 6, 0.1, 4)
    nan.A[5, 1] = np.nan
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(nan.A), nan.p)
    assert e.value.code == ils.ILS_ERR_NONFINITE
    ok = W.dense_gaussian(60, 10, 6, 0.1, 5)
    ok.b[3] = np.inf
    import torch
    s = ils.Solver(colmajor(ok.A), ok.p)
    x = vec(np.zeros(6))
    info = s.solve(vec(ok.b), x, tol=1e-12, allow=(ils.ILS_ERR_NONFINITE,))
    assert info.status == ils.ILS_ERR_NONFINITE
    s.close()


def test_many_rhs_wide_path_matches_oracle(ils):
    """40 right-hand sides in one call take the GEMM-based path (all columns per step); each
    column matches the oracle to 1e-10 and the 8-column passes to 1e-12, with a warm start
    that is already converged for one column (it returns x0 after zero steps)."""
    import torch
    inst = W.dense_gaussian(1600, 400, 120, 0.3, 21)
    rng = np.random.default_rng(5)
    k = 40
    Bm = inst.A @ rng.standard_normal((inst.n, k)) + 1e-3 * rng.standard_normal((inst.m, k))
    Xs = O.normal_equation_solve(inst.A, Bm, inst.p)
    s = ils.Solver(colmajor(inst.A), inst.p)
    Bt = colmajor(Bm)
    Xw = torch.zeros((k, inst.n), dtype=torch.float64, device="cuda")
    info = s.solve_many(Bt, Xw, tol=1e-12)
    Xn = torch.zeros((k, inst.n), dtype=torch.float64, device="cuda")
    for c0 in range(0, k, 8):
        s.solve_many(Bt[c0:c0 + 8], Xn[c0:c0 + 8], tol=1e-12)
    torch.cuda.synchronize()
    xw, xn = to_np_colmajor(Xw), to_np_colmajor(Xn)
    assert info.status == ils.ILS_OK
    for c in range(k):
        assert relerr(xw[:, c], Xs[:, c]) <= 1e-10
        assert relerr(xw[:, c], xn[:, c]) <= 1e-12
    X0 = torch.zeros((k, inst.n), dtype=torch.float64, device="cuda")
    X0[3] = torch.from_numpy(Xs[:, 3]).cuda()
    info2 = s.solve_many(Bt, X0, x0_zero=False, tol=1e-10)
    torch.cuda.synchronize()
    assert info2.status == ils.ILS_OK
    assert np.array_equal(X0[3].cpu().numpy(), Xs[:, 3])
    s.close()
