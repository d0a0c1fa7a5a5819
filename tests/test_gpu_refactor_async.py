"""GPU: ils_refactor_async (setup enqueued without a wait; the next solve reports its status).

The asynchronous path must give exactly the results of ils_refactor + ils_solve (the same
kernels on the same data; A^T J b may run on a second stream), report a failed setup at the
solve, and settle a failed FP32 pivot test by the FP64 factorization before solving again.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import colmajor, relerr, vec

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


def _solve(ils, s, At, b, refactor_async, allow=None):
    import torch
    x = vec(np.zeros(s.n))
    (s.refactor_async if refactor_async else s.refactor)(At)
    kw = {} if allow is None else {"allow": allow}
    info = s.solve(b, x, tol=1e-12, **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_async_matches_sync(ils, prec):
    precision = {"fp64": ils.ILS_FP64, "fp32": ils.ILS_FP32_REFINE, "bf16": ils.ILS_BF16_REFINE}[prec]
    inst = W.config2() if prec != "fp64" else W.config1()
    other = W.dense_gaussian(inst.p, inst.q, inst.n, 0.25, 77)  # a different A of the same shape
    At, At2 = colmajor(inst.A), colmajor(other.A)
    b, b2 = vec(inst.b), vec(other.b)
    s = ils.Solver(At2, inst.p, ils.options(precision=precision, timing=1))
    x_sync, info_sync = _solve(ils, s, At, b, False)
    _solve(ils, s, At2, b2, True)  # an async setup of another matrix in between
    x_async, info_async = _solve(ils, s, At, b, True)
    assert np.array_equal(x_sync, x_async)
    assert info_sync.status == info_async.status == ils.ILS_OK
    assert info_sync.outer_iters == info_async.outer_iters
    assert relerr(x_async, O.qr_cholesky_solve(inst.A, inst.b, inst.p)) <= 1e-10
    assert s.timings()["setup"] > 0.0
    s.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_async_reports_failed_setup_at_solve(ils, prec):
    """A^T J A indefinite: the asynchronous setup returns OK, the solve reports NOT_SPD."""
    good = W.dense_gaussian(400, 300, 60, 0.3, 3)
    bad = W.dense_gaussian(400, 300, 60, 2.0, 3)
    assert not O.is_spd(O.normal_matrix(bad.A, bad.p))
    s = ils.Solver(colmajor(good.A), good.p, ils.options(precision=prec))
    Abad, bbad = colmajor(bad.A), vec(bad.b)  # in place before the asynchronous setup
    s.refactor_async(Abad)
    x = vec(np.zeros(good.n))
    with pytest.raises(ils.ILSError) as e:
        s.solve(bbad, x, tol=1e-12)
    assert e.value.code == ils.ILS_ERR_NOT_SPD
    # the handle recovers with a valid matrix
    x2, info = _solve(ils, s, colmajor(good.A), vec(good.b), True)
    assert info.status == ils.ILS_OK
    assert relerr(x2, O.qr_cholesky_solve(good.A, good.b, good.p)) <= 1e-10
    s.close()


def test_async_fp32_pivot_failure_settled_in_fp64(ils):
    """An entry of A_1^T A_1 beyond the FP32 range: the FP32 inverse fails, the solve runs the
    FP64 factorization, forms P and B from it and solves again."""
    inst = W.dense_gaussian(300, 240, 40, 0.3, 11)
    A = inst.A.copy()
    A[: inst.p, 0] *= 2.0 ** 64
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE))
    x, info = _solve(ils, s, colmajor(A), vec(inst.b), True,
                     allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    x_sync, info_sync = _solve(ils, s, colmajor(A), vec(inst.b), False,
                               allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    assert info.status == info_sync.status
    assert np.array_equal(x, x_sync)
    s.close()


def test_deferred_b_reaches_the_paths_that_read_it(ils):
    """With FP32 refinement the asynchronous setup leaves B = P Abar2 to be formed after the
    one-cluster solve (which does not read it).  A multi-column solve reads B: after a setup
    of a second matrix it must see that matrix's B, so its answers equal, bit for bit, those
    of a handle set up on that matrix alone."""
    import torch
    inst = W.config2()
    other = W.dense_gaussian(inst.p, inst.q, inst.n, 0.25, 78)
    At, At2 = colmajor(inst.A), colmajor(other.A)
    k = 4
    Bm = np.stack([inst.b * (1.0 + 0.25 * c) for c in range(k)], axis=1)
    opts = ils.options(precision=ils.ILS_FP32_REFINE)
    s = ils.Solver(At2, inst.p, opts)
    x0 = vec(np.zeros(inst.n))
    s.solve(vec(other.b), x0, tol=1e-12)  # one column: the cluster solve, then B behind it
    Bdev = colmajor(Bm)  # in place before the asynchronous setup
    s.refactor_async(At)
    X = colmajor(np.zeros((inst.n, k)))
    info = s.solve_many(Bdev, X, tol=1e-12)
    ref = ils.Solver(At, inst.p, opts)
    Xr = colmajor(np.zeros((inst.n, k)))
    info_r = ref.solve_many(colmajor(Bm), Xr, tol=1e-12)
    torch.cuda.synchronize()
    assert info.status == info_r.status == ils.ILS_OK
    assert info.outer_iters == info_r.outer_iters
    assert torch.equal(X, Xr)
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    assert relerr(X.cpu().numpy()[0], xs) <= 1e-10
    s.close()
    ref.close()
