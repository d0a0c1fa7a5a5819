"""FP64 oracle of the ILS products for a sparse A stored in CSR (test infrastructure only).

The paper's methods (Alg. 1, 2 and 5) only ever touch A through A_1^T A_1, A_2^T A_2,
A^T J b and single columns of A_1 (Sec. 2-4); a sparse A changes how those are
formed, not what they are.  This module forms them from the CSR arrays with
scipy.sparse (a library primitive standing in for the matrix products) and solves
the normal equations (1.2) by Cholesky of H = A^T J A.  For tiny inputs
:func:`csr_dense` rebuilds the dense matrix so that the dense oracle applies.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline may
call this module.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sps

__all__ = ["csr_matrix", "csr_dense", "sparse_gram_blocks", "sparse_rhs_bar", "sparse_residual",
           "sparse_relres", "sparse_normal_solve", "column_counts"]


def csr_matrix(m, n, rowptr, colind, val):
    return sps.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(colind), np.asarray(rowptr)),
                          shape=(m, n))


def csr_dense(m, n, rowptr, colind, val):
    """The dense m x n matrix the CSR arrays describe, one stored entry at a time."""
    A = np.zeros((m, n))
    for r in range(m):
        for e in range(int(rowptr[r]), int(rowptr[r + 1])):
            A[r, int(colind[e])] += float(val[e])
    return A


def sparse_gram_blocks(m, n, p, rowptr, colind, val):
    """Abar1 = A_1^T A_1 and Abar2 = A_2^T A_2 (Sec. 2), dense n x n."""
    A = csr_matrix(m, n, rowptr, colind, val)
    A1, A2 = A[:p], A[p:]
    return (A1.T @ A1).toarray(), (A2.T @ A2).toarray()


def sparse_rhs_bar(m, n, p, rowptr, colind, val, b):
    """bbar = A^T J b = A_1^T b_1 - A_2^T b_2 (Alg. 1 step 4)."""
    A = csr_matrix(m, n, rowptr, colind, val)
    b = np.asarray(b, dtype=np.float64)
    return A[:p].T @ b[:p] - A[p:].T @ b[p:]


def sparse_residual(m, n, p, rowptr, colind, val, b, x):
    """A^T J (b - A x), block-wise as A_1^T(b_1 - A_1 x) - A_2^T(b_2 - A_2 x)."""
    A = csr_matrix(m, n, rowptr, colind, val)
    b = np.asarray(b, dtype=np.float64)
    r = b - A @ x
    return A[:p].T @ r[:p] - A[p:].T @ r[p:]


def sparse_relres(m, n, p, rowptr, colind, val, b, x):
    """||A^T J (b - A x)|| / ||A^T J b||, the square root of the paper's RR (Sec. 5)."""
    r = sparse_residual(m, n, p, rowptr, colind, val, b, x)
    return float(np.linalg.norm(r) / np.linalg.norm(sparse_rhs_bar(m, n, p, rowptr, colind, val, b)))


def sparse_normal_solve(m, n, p, rowptr, colind, val, b):
    """x* = H^{-1} A^T J b with H = Abar1 - Abar2 factored by Cholesky (eq. (1.2)).

    The error of this route is about kappa(H) u; the sparse workloads have kappa(H)
    near 2, so it is accurate to a few units of rounding there.  Raises
    numpy.linalg.LinAlgError when H is not SPD (condition (1.3)).
    """
    G1, G2 = sparse_gram_blocks(m, n, p, rowptr, colind, val)
    H = G1 - G2
    c, low = sla.cho_factor(H, lower=True)
    if not np.all(np.isfinite(c)):
        raise np.linalg.LinAlgError("H is not SPD")
    return sla.cho_solve((c, low), sparse_rhs_bar(m, n, p, rowptr, colind, val, b)), H


def column_counts(m, n, p, rowptr, colind):
    """Entries per column of A, and of A_1 alone."""
    colind = np.asarray(colind)
    rows = np.repeat(np.arange(m), np.diff(np.asarray(rowptr)))
    return np.bincount(colind, minlength=n), np.bincount(colind[rows < p], minlength=n)
