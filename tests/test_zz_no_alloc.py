"""ils_gram_noalloc: the Gram product for callers that cannot allocate device memory.

Such callers (code under stream capture with allocation forbidden, plugins whose host
application owns the device allocator) get C = X^T X with the split-K partial sums in
the library's fixed device array.  This test compares two consecutive calls with the
regular path (ils_setup with q = 0, then ils_get_matrix of A_1^T A_1), within the FP64
product error bound the other Gram tests use.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from tests.helpers import colmajor, gemm_bound, to_np_colmajor

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


def regular_gram(ils, X):
    import torch
    K, n = X.shape
    s = ils.Solver(colmajor(X), K)  # p = K, q = 0: A_1 = X
    out = torch.empty((n, n), dtype=torch.float64, device="cuda")
    s.get_matrix(ils.MAT_GRAM1, out)
    torch.cuda.synchronize()
    s.close()
    return to_np_colmajor(out)


def noalloc_gram(ils, X):
    import torch
    K, n = X.shape
    Xd = colmajor(X)
    C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = ils.lib().ils_gram_noalloc(K, n, Xd.data_ptr(), Xd.stride(0), C.data_ptr(), C.stride(0), stream)
    assert code == ils.ILS_OK, ils.status_string(code)
    torch.cuda.synchronize()
    return to_np_colmajor(C)


@pytest.mark.parametrize("K,n", [(16000, 500), (3001, 257), (70, 33), (20000, 1024)])
def test_noalloc_gram_matches_regular_path_twice(ils, K, n):
    rng = np.random.default_rng(K + n)
    for call in range(2):
        X = rng.standard_normal((K, n)) * (1.0 + call)
        ref = regular_gram(ils, X)
        got = noalloc_gram(ils, X)
        bound = gemm_bound(X, X)
        assert np.all(np.abs(got - ref) <= 2 * bound), call
        assert np.array_equal(got, got.T)


def test_noalloc_rejects_sizes_beyond_its_scratch(ils):
    code = ils.lib().ils_gram_noalloc(10, 1025, 1, 10, 1, 1025, None)
    assert code == ils.ILS_ERR_INVALID_ARG


def test_noalloc_empty_reduction_gives_zero(ils):
    """K = 0: X^T X is the n x n zero matrix, written in full (over a NaN-filled C), twice."""
    import torch
    for _ in range(2):
        n = 40
        C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        code = ils.lib().ils_gram_noalloc(0, n, None, 1, C.data_ptr(), C.stride(0), stream)
        assert code == ils.ILS_OK
        torch.cuda.synchronize()
        assert torch.count_nonzero(C).item() == 0
