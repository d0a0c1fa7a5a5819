"""Seeded synthetic inputs for the indefinite least squares (ILS) solver.

This module only draws random numbers and arranges them into the shapes of the
paper's workloads and of the five evaluation configurations; it holds none of the
solver's arithmetic.  Both the CPU oracle and the CUDA path read the arrays made
here, so a test always hands the two sides identical bytes.

Layout conventions (shared with the C-ABI):
  * ``A`` is an m x n float64 array in column-major (Fortran) order; rows
    ``0..p-1`` form ``A_1`` (the ``+I_p`` block of J) and rows ``p..m-1`` form
    ``A_2`` (the ``-I_q`` block), as in the partition of Sec. 1.4, eq. (1.4).
  * ``b`` is a length-m vector, or an m x k column-major matrix of k right-hand
    sides.

All generators use ``numpy.random.default_rng`` (PCG64) and draw in a fixed
order: A_1, A_2, x_true, noise.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Instance",
    "SparseInstance",
    "dense_gaussian",
    "config1",
    "config2",
    "config2_roofline",
    "config3_sparse",
    "config4_batched",
    "config4_shapes",
    "config5_warmstart",
    "paper_table_workload",
    "tiny_integer_instance",
    "mp_scale",
]


@dataclass
class Instance:
    """One dense ILS instance ``min (b-Ax)^T J (b-Ax)``, J = diag(I_p, -I_q)."""

    A: np.ndarray  # (m, n) float64, Fortran order
    b: np.ndarray  # (m,) or (m, k) float64, Fortran order
    p: int
    q: int
    x_true: np.ndarray  # the vector(s) used to build b (not the ILS solution)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


@dataclass
class SparseInstance:
    """A sparse ILS instance stored as CSR (row pointers, column indices, values)."""

    m: int
    n: int
    p: int
    q: int
    rowptr: np.ndarray  # (m+1,) int32
    colind: np.ndarray  # (nnz,) int32
    val: np.ndarray  # (nnz,) float64
    b: np.ndarray  # (m,) float64
    x_true: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])


def mp_scale(p: int, q: int, n: int) -> float:
    """Scale for A_2 so that A^T J A stays SPD with margin.

    With i.i.d. N(0,1) blocks the Marchenko-Pastur edges give
    sigma_min(A_1) ~ sqrt(p) - sqrt(n) and sigma_max(A_2) ~ sqrt(q) + sqrt(n);
    scaling A_2 by half their ratio keeps sigma_max(s A_2) near sigma_min(A_1)/2.
    """
    return 0.5 * (math.sqrt(p) - math.sqrt(n)) / (math.sqrt(q) + math.sqrt(n))


def _stack(A1: np.ndarray, A2: np.ndarray) -> np.ndarray:
    A = np.empty((A1.shape[0] + A2.shape[0], A1.shape[1]), dtype=np.float64, order="F")
    A[: A1.shape[0]] = A1
    A[A1.shape[0]:] = A2
    return A


def dense_gaussian(p: int, q: int, n: int, a2_scale: float, seed, k: int = 1,
                   noise: float = 1e-3, name: str = "") -> Instance:
    """A_1 ~ N(0,1)^{p x n}, A_2 ~ a2_scale * N(0,1)^{q x n}, b = A x + noise * N(0,1).

    ``k`` right-hand sides are drawn as one n x k block of x and one m x k block
    of noise.  For k == 1 ``b`` and ``x_true`` are vectors.
    """
    rng = np.random.default_rng(seed)
    A1 = rng.standard_normal((p, n))
    A2 = a2_scale * rng.standard_normal((q, n)) if q > 0 else np.zeros((0, n))
    A = _stack(A1, A2)
    m = p + q
    if k == 1:
        x = rng.standard_normal(n)
        e = rng.standard_normal(m)
        b = A @ x + noise * e
    else:
        x = np.asfortranarray(rng.standard_normal((n, k)))
        e = rng.standard_normal((m, k))
        b = np.asfortranarray(A @ x + noise * e)
    return Instance(A=A, b=b, p=p, q=q, x_true=x, name=name,
                    meta={"seed": seed, "a2_scale": a2_scale, "k": k})


def config1() -> Instance:
    """Small dense case: A_1 400x50, A_2 0.2*N(0,1) 100x50, seed 0."""
    return dense_gaussian(400, 100, 50, 0.2, 0, name="dense 500x50 (p=400, q=100)")


def config2(k: int = 1) -> Instance:
    """Large dense single-RHS case: A_1 16000x500, A_2 0.3*N(0,1) 4000x500, seed 1."""
    return dense_gaussian(16000, 4000, 500, 0.3, 1, k=k,
                          name="dense 20000x500 (p=16000, q=4000)")


def config2_roofline(q: int = 262144) -> Instance:
    """Bandwidth case: A_1 16000x500 and a tall A_2 (q x 500) far larger than L2."""
    p, n = 16000, 500
    return dense_gaussian(p, q, n, mp_scale(p, q, n), 1,
                          name=f"dense {p + q}x{n} (p={p}, q={q})")


def config3_sparse(m: int = 100000, n: int = 2000, p: int = 80000, density: float = 0.005,
                   a2_scale: float = 0.25, seed: int = 3, noise: float = 1e-3) -> SparseInstance:
    """Sparse case: each entry present independently with probability ``density``.

    The Bernoulli pattern over the row-major flattened m x n grid is drawn as a
    sequence of geometric gaps (the exact law of a Bernoulli process); values are
    N(0,1) and rows p..m-1 (the A_2 block) are scaled by ``a2_scale``.
    """
    rng = np.random.default_rng(seed)
    total = m * n
    expect = int(total * density)
    gaps = rng.geometric(density, size=expect + 8 * int(math.sqrt(expect) + 16))
    pos = np.cumsum(gaps) - 1
    while pos[-1] < total:  # extremely unlikely; extend the process
        more = rng.geometric(density, size=1024)
        pos = np.concatenate([pos, pos[-1] + np.cumsum(more)])
    pos = pos[pos < total]
    rows = (pos // n).astype(np.int64)
    cols = (pos % n).astype(np.int32)
    val = rng.standard_normal(pos.shape[0])
    val[rows >= p] *= a2_scale
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    x = rng.standard_normal(n)
    e = rng.standard_normal(m)
    # b = A x + noise: one dot product per stored row.
    b = np.bincount(rows, weights=val * x[cols], minlength=m) + noise * e
    return SparseInstance(m=m, n=n, p=p, q=m - p, rowptr=rowptr, colind=cols, val=val,
                          b=b, x_true=x, name=f"sparse {m}x{n} density {density}")


def config4_shapes(count: int = 256, seed: int = 4):
    """The (m, n, p, q) of the batched workload, without drawing the matrices."""
    shapes = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        n = int(rng.integers(32, 513))
        m = int(round(rng.uniform(4.0, 20.0) * n))
        q = int(round(rng.uniform(0.05, 0.25) * m))
        shapes.append((m, n, m - q, q))
    return shapes


def config4_batched(count: int = 256, k: int = 8, seed: int = 4, indices=None):
    """Batched uneven instances: n ~ U{32..512}, m = round(U[4,20] n), q = round(U[.05,.25] m).

    Instance i draws from ``default_rng([seed, i])``: first its shape, then A_1,
    A_2 (scaled by :func:`mp_scale`), the n x k block of x and the noise.
    """
    out = []
    idx = range(count) if indices is None else indices
    for i in idx:
        rng = np.random.default_rng([seed, i])
        n = int(rng.integers(32, 513))
        m = int(round(rng.uniform(4.0, 20.0) * n))
        q = int(round(rng.uniform(0.05, 0.25) * m))
        p = m - q
        s = mp_scale(p, q, n)
        A1 = rng.standard_normal((p, n))
        A2 = s * rng.standard_normal((q, n))
        A = _stack(A1, A2)
        x = np.asfortranarray(rng.standard_normal((n, k)))
        e = rng.standard_normal((m, k))
        b = np.asfortranarray(A @ x + 1e-3 * e)
        out.append(Instance(A=A, b=b, p=p, q=q, x_true=x, name=f"batched[{i}] {m}x{n}",
                            meta={"index": i, "a2_scale": s, "k": k}))
    return out


@dataclass
class WarmStartFamily:
    """Parametric right-hand sides b(theta) = F theta + noise for one fixed A."""

    A: np.ndarray  # (m, n) Fortran
    p: int
    q: int
    F: np.ndarray  # (m, d) feature matrix
    noise: float
    seed: int

    def thetas(self, count: int, seed: int) -> np.ndarray:
        """``count`` parameter vectors theta ~ U[-1,1]^d, as a (count, d) array."""
        rng = np.random.default_rng(seed)
        return rng.uniform(-1.0, 1.0, size=(count, self.F.shape[1]))

    def rhs(self, thetas: np.ndarray, seed: int, start: int = 0) -> np.ndarray:
        """b for each theta row, as an m x count Fortran array.

        The noise for sample ``start + j`` comes from ``default_rng([seed, start + j])``
        so any slice of a long list of samples can be rebuilt on its own.
        """
        m = self.A.shape[0]
        cnt = thetas.shape[0]
        B = np.empty((m, cnt), dtype=np.float64, order="F")
        for j in range(cnt):
            e = np.random.default_rng([seed, start + j]).standard_normal(m)
            B[:, j] = self.F @ thetas[j] + self.noise * e
        return B


def config5_warmstart(p: int = 6144, q: int = 2048, n: int = 256, d: int = 16,
                      a2_scale: float = 0.25, seed: int = 5) -> WarmStartFamily:
    """Fixed A (A_1 6144x256, A_2 0.25*N(0,1) 2048x256) and F ~ N(0,1)^{8192x16}."""
    rng = np.random.default_rng(seed)
    A1 = rng.standard_normal((p, n))
    A2 = a2_scale * rng.standard_normal((q, n))
    F = rng.standard_normal((p + q, d))
    return WarmStartFamily(A=_stack(A1, A2), p=p, q=q, F=F, noise=1e-3, seed=seed)


def paper_table_workload(p: int, q: int, n: int, seed: int = 0, diag: float = 7.0) -> Instance:
    """The shape of the paper's experiments (Sec. 5.2, Tables 2-5).

    A_1 = U[0,1)^{p x n}, A_2 = diag * (the q x n matrix with ones on its main
    diagonal), b_1 = U[0,1)^p, b_2 = U[0,1)^q.  The paper uses diag = 7; a
    reduced-size replay may lower it so that rho(Abar1^{-1} Abar2) matches the
    paper's size (lambda_min(Abar1) grows with p while diag^2 does not).
    """
    rng = np.random.default_rng(seed)
    A1 = rng.random((p, n))
    A2 = np.zeros((q, n))
    d = min(q, n)
    A2[np.arange(d), np.arange(d)] = diag
    b = np.concatenate([rng.random(p), rng.random(q)])
    return Instance(A=_stack(A1, A2), b=b, p=p, q=q, x_true=np.zeros(n),
                    name=f"paper-shape {p + q}x{n} (p={p}, q={q})")


def tiny_integer_instance(p: int, q: int, n: int, seed: int, lo: int = -3, hi: int = 3) -> Instance:
    """Small integer-valued A and b, for exact rational checks (n <= 4)."""
    rng = np.random.default_rng(seed)
    A1 = rng.integers(lo, hi + 1, size=(p, n)).astype(np.float64)
    A2 = rng.integers(-1, 2, size=(q, n)).astype(np.float64)
    b = rng.integers(lo, hi + 1, size=p + q).astype(np.float64)
    return Instance(A=_stack(A1, A2), b=b, p=p, q=q, x_true=np.zeros(n), name="tiny-int")
