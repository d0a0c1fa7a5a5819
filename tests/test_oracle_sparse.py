"""Pins of the sparse-A oracle (CPU): literal products, the dense oracle, generator statistics."""
import math

import numpy as np
import pytest

import oracle as O
import oracle.sparse as OS
import workloads as W

# A = [[1, 0, 2], [0, 3, 0], [4, 0, 1], [0, -1, 1]] with p = 3 (A_2 = last row).
LIT_ROWPTR = np.array([0, 2, 3, 5, 7], dtype=np.int32)
LIT_COLIND = np.array([2, 0, 1, 0, 2, 2, 1], dtype=np.int32)  # unsorted within rows on purpose
LIT_VAL = np.array([2.0, 1.0, 3.0, 4.0, 1.0, 1.0, -1.0])


def test_literal_matrix_products():
    A = OS.csr_dense(4, 3, LIT_ROWPTR, LIT_COLIND, LIT_VAL)
    assert np.array_equal(A, [[1, 0, 2], [0, 3, 0], [4, 0, 1], [0, -1, 1]])
    G1, G2 = OS.sparse_gram_blocks(4, 3, 3, LIT_ROWPTR, LIT_COLIND, LIT_VAL)
    # A_1^T A_1 by hand: columns (1,0,4), (0,3,0), (2,0,1)
    assert np.array_equal(G1, [[17, 0, 6], [0, 9, 0], [6, 0, 5]])
    assert np.array_equal(G2, [[0, 0, 0], [0, 1, -1], [0, -1, 1]])
    b = np.array([1.0, 2.0, 3.0, 4.0])
    # A_1^T b_1 = (1+12, 6, 2+3) = (13, 6, 5); A_2^T b_2 = (0, -4, 4)
    assert np.array_equal(OS.sparse_rhs_bar(4, 3, 3, LIT_ROWPTR, LIT_COLIND, LIT_VAL, b), [13, 10, 1])
    total, a1 = OS.column_counts(4, 3, 3, LIT_ROWPTR, LIT_COLIND)
    assert list(total) == [2, 2, 3] and list(a1) == [2, 1, 2]


def test_literal_solve_is_exact():
    b = np.array([1.0, 2.0, 3.0, 4.0])
    x, H = OS.sparse_normal_solve(4, 3, 3, LIT_ROWPTR, LIT_COLIND, LIT_VAL, b)
    A = OS.csr_dense(4, 3, LIT_ROWPTR, LIT_COLIND, LIT_VAL)
    exact = O.exact_solve_fraction(A, b, 3)
    assert np.max(np.abs(x - np.array([float(v) for v in exact]))) < 1e-14
    assert OS.sparse_relres(4, 3, 3, LIT_ROWPTR, LIT_COLIND, LIT_VAL, b, x) < 1e-14


@pytest.fixture(scope="module")
def small():
    return W.config3_sparse(m=2000, n=60, p=1600, density=0.05, seed=33)


def test_sparse_products_match_dense_oracle(small):
    s = small
    A = OS.csr_dense(s.m, s.n, s.rowptr, s.colind, s.val)
    G1, G2 = OS.sparse_gram_blocks(s.m, s.n, s.p, s.rowptr, s.colind, s.val)
    D1, D2 = O.gram_blocks(A, s.p)
    assert np.max(np.abs(G1 - D1)) <= 1e-12 * np.max(np.abs(D1))
    assert np.max(np.abs(G2 - D2)) <= 1e-12 * np.max(np.abs(D2))
    bb = OS.sparse_rhs_bar(s.m, s.n, s.p, s.rowptr, s.colind, s.val, s.b)
    assert np.max(np.abs(bb - O.rhs_bar(A, s.b, s.p))) <= 1e-12 * np.max(np.abs(bb))
    x, _ = OS.sparse_normal_solve(s.m, s.n, s.p, s.rowptr, s.colind, s.val, s.b)
    xq = O.qr_cholesky_solve(A, s.b, s.p)
    assert np.linalg.norm(x - xq) <= 1e-12 * np.linalg.norm(xq)
    # the generator's b is A x_true plus 1e-3 noise
    assert np.linalg.norm(s.b - A @ s.x_true) < 5e-3 * math.sqrt(s.m)


def test_generator_pattern_and_scaling(small):
    s = small
    rows = np.repeat(np.arange(s.m), np.diff(s.rowptr))
    nnz = s.val.size
    expect = s.m * s.n * 0.05
    assert abs(nnz - expect) < 5 * math.sqrt(expect)
    # no duplicate (row, column) pairs; columns sorted within rows (gap process)
    key = rows.astype(np.int64) * s.n + s.colind
    assert np.all(np.diff(key) > 0)
    assert abs(np.std(s.val[rows < s.p]) - 1.0) < 0.05
    assert abs(np.std(s.val[rows >= s.p]) - 0.25) < 0.02


def test_full_size_sparse_instance_is_spd():
    """The 100000 x 2000 (density 0.005) instance: H = A^T J A is SPD (Cholesky succeeds)."""
    s = W.config3_sparse()
    assert (s.m, s.n, s.p) == (100000, 2000, 80000)
    assert abs(s.val.size - 1.0e6) < 5 * 1000
    x, H = OS.sparse_normal_solve(s.m, s.n, s.p, s.rowptr, s.colind, s.val, s.b)
    ev = np.linalg.eigvalsh(H)
    assert ev[0] > 0.0
    total, a1 = OS.column_counts(s.m, s.n, s.p, s.rowptr, s.colind)
    assert total.max() <= 4096
    assert np.linalg.norm(x - s.x_true) < 1e-2 * np.linalg.norm(s.x_true)
