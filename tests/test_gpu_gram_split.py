"""GPU parity of the tensor-core split Gram (options.gram = ILS_GRAM_SPLIT).

A_1^T A_1 and A_2^T A_2 built from exact BF16 slice products must meet the FP64
product bound 4 K u |A|^T |A| elementwise against the oracle's FP64 Gram, and SP on
top of them must reach ||x - x*|| / ||x*|| <= 1e-10 (Alg. 1 with Sec. 5's stop).
"""
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


# (p, q, n): a single 64-row K stage, ragged tiles, two K chunks, several tiles.
SHAPES = [(64, 16, 8), (128, 40, 128), (100, 30, 33), (3001, 499, 257), (16000, 4000, 500), (20000, 100, 130)]


@pytest.mark.parametrize("p,q,n", SHAPES)
def test_split_gram_meets_fp64_bound(ils, p, q, n):
    import torch
    s_ = 0.3 * min(1.0, (p ** 0.5 - n ** 0.5) / (q ** 0.5 + n ** 0.5))
    inst = W.dense_gaussian(p, q, n, s_, 7000 + n)
    s = ils.Solver(colmajor(inst.A), p, ils.options(gram=ils.ILS_GRAM_SPLIT, route=ils.ILS_ROUTE_EXPLICIT))
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    A1, A2 = inst.A[:p], inst.A[p:]
    G1o, G2o = O.gram_blocks(inst.A, p)
    s.get_matrix(ils.MAT_GRAM1, out)
    G1 = to_np_colmajor(out)
    assert np.all(np.abs(G1 - G1o) <= gemm_bound(A1, A1)), np.max(np.abs(G1 - G1o) / gemm_bound(A1, A1))
    assert np.array_equal(G1, G1.T)
    s.get_matrix(ils.MAT_GRAM2, out)
    G2 = to_np_colmajor(out)
    assert np.all(np.abs(G2 - G2o) <= gemm_bound(A2, A2) + 1e-300)
    # The split keeps 50 bits below each column's scale: far inside the FP64 bound.
    scale = np.max(np.abs(A1), axis=0)
    tight = 64 * p * 2.0 ** -50 * np.outer(scale, scale)
    assert np.all(np.abs(G1 - G1o) <= tight)
    s.close()


def test_split_gram_sp_solves(ils):
    for inst in (W.config1(), W.config2()):
        xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
        s = ils.Solver(colmajor(inst.A), inst.p, ils.options(gram=ils.ILS_GRAM_SPLIT))
        x = vec(np.zeros(inst.n))
        info = s.solve(vec(inst.b), x, tol=1e-12)
        assert info.status == ils.ILS_OK
        assert relerr(x.cpu().numpy(), xs) <= 1e-10
        s.close()


def test_split_gram_nonfinite_input(ils):
    inst = W.dense_gaussian(200, 20, 16, 0.2, 3)
    inst.A[7, 3] = np.inf
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(inst.A), inst.p, ils.options(gram=ils.ILS_GRAM_SPLIT))
    assert e.value.code == ils.ILS_ERR_NONFINITE
