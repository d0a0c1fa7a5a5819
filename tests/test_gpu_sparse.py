"""GPU parity of the sparse-A path (ils_setup_csr) against the CPU oracle.

Small instances (2000 x 60 at density 0.05, a few hundred entries per column, so each
column spans many threads of a chain and the pattern is ragged) are checked against
the dense oracle on the densified matrix: the setup Grams element by element, every
method's solution against the QR-Cholesky x*, and one SP-RK-RGS outer iteration step
by step (both sides draw the same Philox indices).  The 100000 x 2000 instance at
density 0.005 is checked against x* from the Cholesky of H (kappa(H) is about 2 there).
"""
import numpy as np
import pytest

import oracle as O
import oracle.sparse as OS
import workloads as W
from tests.helpers import gemm_bound, relerr, to_np_colmajor, vec

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


def csr_dev(rowptr, colind, val):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(rowptr, dtype=np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(colind, dtype=np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(val, dtype=np.float64)).cuda())


def make(ils, inst, **opt):
    return ils.Solver.from_csr(inst.m, inst.n, inst.p, *csr_dev(inst.rowptr, inst.colind, inst.val),
                               ils.options(**opt))


def solve(ils, s, b, tol=1e-12):
    import torch
    x = vec(np.zeros(s.n))
    info = s.solve(vec(b), x, tol=tol, allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.fixture(scope="module")
def small():
    inst = W.config3_sparse(m=2000, n=60, p=1600, density=0.05, seed=33)
    A = OS.csr_dense(inst.m, inst.n, inst.rowptr, inst.colind, inst.val)
    return inst, A, O.qr_cholesky_solve(A, inst.b, inst.p)


def test_sparse_setup_grams(ils, small):
    import torch
    inst, A, _ = small
    s = make(ils, inst)
    n = inst.n
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    for which, (X, ref) in enumerate([(A[:inst.p], None), (A[inst.p:], None)]):
        s.get_matrix(which, out)
        torch.cuda.synchronize()
        G = to_np_colmajor(out)
        ref = X.T @ X
        assert np.all(np.abs(G - ref) <= gemm_bound(X, X) + 1e-300), which
        assert np.array_equal(G, G.T)
    s.close()


@pytest.mark.parametrize("method", ["sp", "rk_rgs", "scd"])
def test_sparse_fp64_methods_converge(ils, small, method):
    inst, A, xs = small
    m = {"sp": ils.ILS_SP, "rk_rgs": ils.ILS_SP_RK_RGS, "scd": ils.ILS_SP_SCD}[method]
    s = make(ils, inst, method=m, seed=5)
    x, info = solve(ils, s, inst.b)
    s.close()
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10, (info.status, relerr(x, xs))
    if method == "rk_rgs":
        _, oinfo = O.sp_rk_rgs_solve(A, inst.b, inst.p, tol=1e-12, seed=5)
        assert abs(info.outer_iters - oinfo.outer_iters) <= 2


@pytest.fixture(scope="module")
def ragged():
    """Sizes that divide by no cluster size: slices and residual shares end ragged."""
    inst = W.config3_sparse(m=2003, n=61, p=1603, density=0.05, seed=34)
    return inst, OS.csr_dense(inst.m, inst.n, inst.rowptr, inst.colind, inst.val)


@pytest.fixture(scope="module")
def long_columns():
    """About 600 entries per column of A_1 (beyond what a lane holds in registers) and
    n = 600 (beyond the residual share a lane holds in registers)."""
    a = W.config3_sparse(m=3600, n=20, p=3000, density=0.2, seed=35)
    b = W.config3_sparse(m=3600, n=600, p=3000, density=0.02, seed=36)
    return [(x, OS.csr_dense(x.m, x.n, x.rowptr, x.colind, x.val)) for x in (a, b)]


def trajectory(ils, inst, A, ctas, steps=300, seed=9):
    s = make(ils, inst, method=ils.ILS_SP_RK_RGS, max_outer=1, max_inner=steps, check_every=10 ** 9, seed=seed,
             chain_ctas=ctas)
    x, info = solve(ils, s, inst.b, tol=0.0)
    s.close()
    xo, oinfo = O.sp_rk_rgs_solve(A, inst.b, inst.p, tol=0.0, max_outer=1, max_inner=steps,
                                  check_every=10 ** 9, seed=seed)
    assert info.inner_iters == steps == oinfo.inner_iters[0]
    assert np.linalg.norm(x - xo) <= 1e-11 * np.linalg.norm(xo), np.linalg.norm(x - xo) / np.linalg.norm(xo)


@pytest.mark.parametrize("ctas", [-1, 1, 2, 4, 8])
def test_sparse_rk_rgs_trajectory_matches_oracle(ils, ragged, ctas):
    """300 inner steps of the first outer iteration, no inner stop test: same picks, same z,
    for one CTA with global vectors and for every cluster size."""
    inst, A = ragged
    trajectory(ils, inst, A, ctas)


@pytest.mark.parametrize("which,ctas", [(0, 1), (0, 2), (1, 1), (1, 8)])
def test_sparse_rk_rgs_trajectory_long_columns(ils, long_columns, which, ctas):
    inst, A = long_columns[which]
    trajectory(ils, inst, A, ctas, steps=200)


@pytest.mark.parametrize("which,ctas", [(0, 1), (1, 1), (1, 2)])
def test_sparse_rk_rgs_fp32_long_columns_converge(ils, long_columns, which, ctas):
    inst, A = long_columns[which]
    xs = O.qr_cholesky_solve(A, inst.b, inst.p)
    s = make(ils, inst, method=ils.ILS_SP_RK_RGS, precision=ils.ILS_FP32_REFINE, seed=8, chain_ctas=ctas)
    x, info = solve(ils, s, inst.b)
    s.close()
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10, (info.status, relerr(x, xs))


@pytest.mark.parametrize("ctas", [-1, 2, 8])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sparse_rk_rgs_cluster_sizes_converge(ils, ragged, ctas, precision):
    inst, A = ragged
    xs = O.qr_cholesky_solve(A, inst.b, inst.p)
    prec = ils.ILS_FP32_REFINE if precision == "fp32" else ils.ILS_FP64
    s = make(ils, inst, method=ils.ILS_SP_RK_RGS, precision=prec, seed=6, chain_ctas=ctas)
    x, info = solve(ils, s, inst.b)
    s.close()
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10, (info.status, relerr(x, xs))


@pytest.mark.parametrize("method", ["sp", "rk_rgs"])
def test_sparse_fp32_refinement(ils, small, method):
    """FP32 inner work with FP64 residuals reaches the FP64 tolerance."""
    inst, _, xs = small
    m = ils.ILS_SP if method == "sp" else ils.ILS_SP_RK_RGS
    s = make(ils, inst, method=m, precision=ils.ILS_FP32_REFINE, seed=2)
    x, info = solve(ils, s, inst.b)
    s.close()
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10, (info.status, relerr(x, xs))
    assert info.refinements >= 1


def test_sparse_many_rhs(ils, small):
    import torch
    inst, A, _ = small
    rng = np.random.default_rng(71)
    k = 3
    Bm = A @ rng.standard_normal((inst.n, k)) + 1e-3 * rng.standard_normal((inst.m, k))
    s = make(ils, inst, method=ils.ILS_SP_RK_RGS, precision=ils.ILS_FP32_REFINE, seed=4)
    Bt = torch.from_numpy(np.ascontiguousarray(Bm.T)).cuda()
    Xt = torch.zeros((k, inst.n), dtype=torch.float64, device="cuda")
    info = s.solve_many(Bt, Xt, tol=1e-12)
    torch.cuda.synchronize()
    s.close()
    X = Xt.cpu().numpy().T
    for c in range(k):
        xs = O.qr_cholesky_solve(A, Bm[:, c], inst.p)
        assert relerr(X[:, c], xs) <= 1e-10, c
    assert info.status == ils.ILS_OK


def test_malformed_csr_is_rejected(ils, small):
    inst, _, _ = small
    bad_col = inst.colind.copy()
    bad_col[17] = inst.n  # out of range
    bad_rowptr = inst.rowptr.copy()
    bad_rowptr[5], bad_rowptr[6] = bad_rowptr[6], bad_rowptr[5] - 1  # decreasing
    dup = inst.colind.copy()
    r = int(np.argmax(np.diff(inst.rowptr) >= 2))
    dup[inst.rowptr[r] + 1] = dup[inst.rowptr[r]]  # the same (row, column) twice
    for rowptr, colind in ((inst.rowptr, bad_col), (bad_rowptr, inst.colind), (inst.rowptr, dup)):
        with pytest.raises(ils.ILSError) as e:
            ils.Solver.from_csr(inst.m, inst.n, inst.p, *csr_dev(rowptr, colind, inst.val), ils.options())
        assert e.value.code == ils.ILS_ERR_INVALID_ARG
    val = inst.val.copy()
    val[3] = np.nan
    with pytest.raises(ils.ILSError) as e:
        ils.Solver.from_csr(inst.m, inst.n, inst.p, *csr_dev(inst.rowptr, inst.colind, val), ils.options())
    assert e.value.code == ils.ILS_ERR_NONFINITE
    # the context is still usable
    s = make(ils, inst)
    s.close()


@pytest.fixture(scope="module")
def full():
    inst = W.config3_sparse()
    xs, _ = OS.sparse_normal_solve(inst.m, inst.n, inst.p, inst.rowptr, inst.colind, inst.val, inst.b)
    return inst, xs


@pytest.mark.parametrize("method,precision", [("rk_rgs", "fp32"), ("rk_rgs", "fp64"), ("scd", "fp64"),
                                              ("sp", "fp64")])
def test_full_size_sparse_solve(ils, full, method, precision):
    """100000 x 2000 CSR at density 0.005: the solution matches x* to 1e-10."""
    inst, xs = full
    m = {"sp": ils.ILS_SP, "rk_rgs": ils.ILS_SP_RK_RGS, "scd": ils.ILS_SP_SCD}[method]
    prec = ils.ILS_FP32_REFINE if precision == "fp32" else ils.ILS_FP64
    s = make(ils, inst, method=m, precision=prec, seed=3)
    x, info = solve(ils, s, inst.b)
    s.close()
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10, (info.status, relerr(x, xs), info.outer_iters)
    r = OS.sparse_relres(inst.m, inst.n, inst.p, inst.rowptr, inst.colind, inst.val, inst.b, x)
    assert r <= 1e-11
