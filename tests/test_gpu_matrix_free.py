"""GPU parity of the matrix-free route: v = A_2^T (A_2 x) streamed in one pass over A_2,
and SP driven by it (x_{k+1} = P (A_2^T A_2 x_k + bbar), Alg. 1 step 6 without Abar2).

Bounds: the FP64-accurate stream (the FP64 copy of an FP64 handle, the double-FP32 copy of a
mixed one) meets 4 q u |A_2|^T |A_2| |x| elementwise; the FP32 copy 1e-5 and the BF16 copy
2e-2 in relative 2-norm; every solve reaches ||x - x*|| / ||x*|| <= 1e-10.
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


@pytest.mark.parametrize("n", [100, 300, 500])
def test_stream_product_parity(ils, n):
    import torch
    p, q = 4 * n, 40 * n + 17
    inst = W.dense_gaussian(p, q, n, W.mp_scale(p, q, n), 60 + n)
    A2 = inst.A[p:]
    x = np.random.default_rng(n).standard_normal(n)
    vo = A2.T @ (A2 @ x)
    for prec, name in ((0, "fp64"), (1, "fp32"), (2, "bf16")):
        precision = {0: ils.ILS_FP64, 1: ils.ILS_FP32_REFINE, 2: ils.ILS_BF16_REFINE}[prec]
        s = ils.Solver(colmajor(inst.A), p, ils.options(precision=precision, route=ils.ILS_ROUTE_MATRIX_FREE))
        v = torch.empty(n, dtype=torch.float64, device="cuda")
        s.aq_product(vec(x), v, prec=0)
        vg = v.cpu().numpy()
        bound = 4 * q * 2.0 ** -53 * (np.abs(A2).T @ (np.abs(A2) @ np.abs(x)))
        assert np.all(np.abs(vg - vo) <= bound), name
        if prec:
            s.aq_product(vec(x), v, prec=prec)
            tol = 1e-5 if prec == 1 else 2e-2
            assert np.linalg.norm(v.cpu().numpy() - vo) <= tol * np.linalg.norm(vo), name
        s.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_matrix_free_solves(ils, precision):
    p, q, n = 2000, 40000, 120
    inst = W.dense_gaussian(p, q, n, W.mp_scale(p, q, n), 77)
    xs = O.normal_equation_solve(inst.A, inst.b, p)
    s = ils.Solver(colmajor(inst.A), p, ils.options(precision=precision, route=ils.ILS_ROUTE_MATRIX_FREE))
    x = vec(np.zeros(n))
    info = s.solve(vec(inst.b), x, tol=1e-12)
    assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), xs) <= 1e-10
    import torch
    with pytest.raises(ils.ILSError):  # Abar2 is never formed on this route
        s.get_matrix(ils.MAT_GRAM2, torch.empty((n, n), dtype=torch.float64, device="cuda"))
    if precision == 0:
        s2 = ils.Solver(colmajor(inst.A), p, ils.options(route=ils.ILS_ROUTE_EXPLICIT))
        x2 = vec(np.zeros(n))
        info2 = s2.solve(vec(inst.b), x2, tol=1e-12)
        assert abs(info.outer_iters - info2.outer_iters) <= 1
        s2.close()
    s.close()


def test_auto_route_choice(ils):
    """An auto-route handle has the A_2 stream exactly when the autotuner chose matrix-free."""
    import torch
    for inst in (W.dense_gaussian(400, 40 * 12 + 1, 12, 0.05, 5), W.config1()):
        s = ils.Solver(colmajor(inst.A), inst.p)
        mf = ils.binding.route_model()["matrix_free"] == 1.0
        v = torch.empty(inst.n, dtype=torch.float64, device="cuda")
        if mf:
            s.aq_product(vec(np.ones(inst.n)), v)
        else:
            with pytest.raises(ils.ILSError):
                s.aq_product(vec(np.ones(inst.n)), v)
        s.close()


def test_tall_bandwidth_configuration(ils):
    """A_1 16000 x 500, A_2 262144 x 500 (A_2 alone 1.05 GB in FP64): mixed precision, BF16 stream."""
    inst = W.config2_roofline()
    xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_BF16_REFINE))
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=1e-12)
    assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), xs) <= 1e-10
    s.close()


def test_route_autotuner_model(ils):
    """route = auto takes the route with the lower modelled cost from measured rates: the
    reported model is consistent with the choice, the rates are positive, config 2 (q = 4000,
    n = 500) in mixed precision stays explicit (in FP64 its A_2^T A_2 on the FP64 pipe costs
    more than streaming A_2), and every choice solves to 1e-10."""
    import torch
    import workloads as W2
    for inst, expect_mf in ((W2.config2(), False), (W2.dense_gaussian(2000, 60000, 64, 0.05, 44), None)):
        for prec in (0, 2):
            s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=prec))
            m = ils.binding.route_model()
            assert m["explicit_s"] > 0 and m["matrix_free_s"] > 0
            assert all(m[k] > 0 for k in ("gram_split_flops", "gram_f64_flops", "bw_fp64", "bw_fp32", "bw_bf16"))
            assert m["matrix_free"] == (1.0 if m["matrix_free_s"] < m["explicit_s"] else 0.0)
            if expect_mf is not None and prec != 0:  # mixed: the split Gram makes Abar2 cheap
                assert m["matrix_free"] == (1.0 if expect_mf else 0.0), (prec, m)
            x = torch.zeros(inst.n, dtype=torch.float64, device="cuda")
            info = s.solve(torch.from_numpy(inst.b).cuda(), x, tol=1e-12)
            torch.cuda.synchronize()
            xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
            assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), xs) <= 1e-10
            s.close()
