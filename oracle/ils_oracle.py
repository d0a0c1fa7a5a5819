"""Plain FP64 restatement of the paper's ILS methods (test infrastructure only).

Notation follows the paper: A = [A_1; A_2] with A_1 p x n and A_2 q x n
(Sec. 1.4, eq. (1.4)), J = diag(I_p, -I_q), Abar1 = A_1^T A_1,
Abar2 = A_2^T A_2, bbar = A^T J b, H = A^T J A = Abar1 - Abar2 (Sec. 2).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline may
call this module.  Nothing here is shared with the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction
import math

import numpy as np
import scipy.linalg as sla

from .philox import step_uniforms

__all__ = [
    "blocks",
    "gram_blocks",
    "rhs_bar",
    "normal_matrix",
    "is_spd",
    "residual",
    "relres",
    "paper_rr",
    "qr_cholesky_solve",
    "normal_equation_solve",
    "exact_solve_fraction",
    "sp_spectral_radius",
    "energy_norm",
    "SolveInfo",
    "sp_solve",
    "column_cumsum",
    "invcdf_pick",
    "scd_rank_from_uniform",
    "rk_step",
    "rgs_step",
    "scd_step",
    "sp_rk_rgs_solve",
    "sp_scd_solve",
    "scd_pick_literal",
    "scd_pick_rank",
    "scd_rank_law",
    "scd_literal_law",
    "scd_fixed_rank_from_uniform",
    "scd_fixed_survival",
    "scd_fixed_rank_law",
    "scd_fixed_literal_law",
    "normal_matrix_condition",
    "error_certificate",
    "sp_rk_rgs_gram_solve",
    "theta_at",
]


# ---------------------------------------------------------------------------
# Problem definition (Sec. 1 and Sec. 2)
# ---------------------------------------------------------------------------

def blocks(A, b, p):
    """Partition of eq. (1.4): A_1 = rows 0..p-1, A_2 = rows p..m-1; same for b."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return A[:p], A[p:], b[:p], b[p:]


def gram_blocks(A, p):
    """Abar1 = A_1^T A_1 and Abar2 = A_2^T A_2 (the split identity of Sec. 2)."""
    A = np.asarray(A, dtype=np.float64)
    A1, A2 = A[:p], A[p:]
    return A1.T @ A1, A2.T @ A2


def rhs_bar(A, b, p):
    """bbar = A^T J b = A_1^T b_1 - A_2^T b_2 (Alg. 1 step 4; Alg. 2 step 3).

    ``b`` may be a vector or an m x k block of right-hand sides.
    """
    A1, A2, b1, b2 = blocks(A, b, p)
    return A1.T @ b1 - A2.T @ b2


def normal_matrix(A, p):
    """H = A^T J A = A_1^T A_1 - A_2^T A_2 (Sec. 2), the matrix of eq. (1.2)."""
    G1, G2 = gram_blocks(A, p)
    return G1 - G2


def is_spd(M) -> bool:
    """Condition (1.3): the normal matrix must be symmetric positive definite."""
    try:
        np.linalg.cholesky(np.asarray(M, dtype=np.float64))
        return True
    except np.linalg.LinAlgError:
        return False


def residual(A, b, p, x):
    """A^T J (b - A x), formed block-wise as A_1^T(b_1 - A_1 x) - A_2^T(b_2 - A_2 x)."""
    A1, A2, b1, b2 = blocks(A, b, p)
    return A1.T @ (b1 - A1 @ x) - A2.T @ (b2 - A2 @ x)


def relres(A, b, p, x):
    """||A^T J (A x - b)||_2 / ||A^T J b||_2: the square root of the paper's RR (Sec. 5).

    For a block of right-hand sides the ratio is taken column by column.
    """
    r = residual(A, b, p, x)
    bb = rhs_bar(A, b, p)
    return np.linalg.norm(r, axis=0) / np.linalg.norm(bb, axis=0)


def paper_rr(A, b, p, x):
    """The paper's stopping quantity RR = ||A^T J (A x - b)||^2 / ||A^T J b||^2 (Sec. 5)."""
    return relres(A, b, p, x) ** 2


def normal_matrix_condition(A, p):
    """kappa_2(H) = lambda_max(H) / lambda_min(H) of H = A^T J A (SPD under (1.3))."""
    lam = np.linalg.eigvalsh(normal_matrix(A, p))
    return float(lam[-1] / lam[0])


def error_certificate(A, b, p, x, kappa=None):
    """kappa(H) * relres(x): an upper bound on ||x - x*|| / ||x*||.

    With r = bbar - H x, x - x* = -H^{-1} r, so ||x - x*|| <= ||H^{-1}|| ||r||; and
    bbar = H x* gives ||x*|| >= ||bbar|| / ||H||.  Dividing, the relative error is at
    most ||H|| ||H^{-1}|| ||r|| / ||bbar|| = kappa_2(H) relres.
    """
    k = normal_matrix_condition(A, p) if kappa is None else kappa
    return k * relres(A, b, p, x)


def energy_norm(v, G):
    """||v||_G = sqrt(v^T G v) for SPD G (notation of Sec. 1.4)."""
    return math.sqrt(float(v @ (G @ v)))


# ---------------------------------------------------------------------------
# Direct solvers: the definition x* = (A^T J A)^{-1} A^T J b
# ---------------------------------------------------------------------------

def qr_cholesky_solve(A, b, p):
    """QR-Cholesky direct method (Sec. 1, after Chandrasekaran et al. 1998).

    A = QR (thin, Q^T Q = I); solve (Q^T J Q) y = Q^T J b by Cholesky; x = R^{-1} y.
    """
    A = np.asarray(A, dtype=np.float64)
    Q, R = np.linalg.qr(A, mode="reduced")
    Q1, Q2 = Q[:p], Q[p:]
    S = Q1.T @ Q1 - Q2.T @ Q2  # Q^T J Q, SPD under (1.3)
    L = np.linalg.cholesky(S)
    b1, b2 = np.asarray(b)[:p], np.asarray(b)[p:]
    QJb = Q1.T @ b1 - Q2.T @ b2
    y = sla.solve_triangular(L.T, sla.solve_triangular(L, QJb, lower=True), lower=False)
    return sla.solve_triangular(R, y, lower=False)


def normal_equation_solve(A, b, p):
    """Cholesky solve of the normal equation (1.2): (A^T J A) x = A^T J b."""
    H = normal_matrix(A, p)
    L = np.linalg.cholesky(H)
    bb = rhs_bar(A, b, p)
    return sla.solve_triangular(L.T, sla.solve_triangular(L, bb, lower=True), lower=False)


def exact_solve_fraction(A, b, p):
    """Exact rational solution of (1.2) by Gaussian elimination over Fractions.

    For small integer-valued inputs only (n <= 4 or so).  Returns a list of Fractions.
    """
    A = [[Fraction(int(round(v))) for v in row] for row in np.asarray(A)]
    bv = [Fraction(int(round(v))) for v in np.asarray(b)]
    m, n = len(A), len(A[0])
    sgn = [1 if i < p else -1 for i in range(m)]
    H = [[sum(sgn[r] * A[r][i] * A[r][j] for r in range(m)) for j in range(n)] for i in range(n)]
    g = [sum(sgn[r] * A[r][i] * bv[r] for r in range(m)) for i in range(n)]
    M = [H[i][:] + [g[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [M[r][j] - f * M[c][j] for j in range(n + 1)]
    return [M[i][n] / M[i][i] for i in range(n)]


def sp_spectral_radius(A, p):
    """rho(Abar1^{-1} Abar2) from the generalized symmetric eigenproblem Abar2 v = lambda Abar1 v.

    Theorem 2.1 states 0 <= lambda < 1 under (1.3).
    """
    G1, G2 = gram_blocks(A, p)
    lam = sla.eigh(G2, G1, eigvals_only=True)
    return float(np.max(np.abs(lam)))


# ---------------------------------------------------------------------------
# Iterative methods
# ---------------------------------------------------------------------------

@dataclass
class SolveInfo:
    outer_iters: int = 0
    inner_iters: list = field(default_factory=list)
    relres: float = float("nan")
    history: list = field(default_factory=list)  # relres of x_0, x_1, ...
    iterates: list = field(default_factory=list)  # x_0, x_1, ... when recorded
    picks: list = field(default_factory=list)  # chosen indices when recorded
    converged: bool = False


def _chol_solve(L, v):
    return sla.solve_triangular(L.T, sla.solve_triangular(L, v, lower=True), lower=False)


def sp_solve(A, b, p, x0=None, tol=1e-12, max_outer=20000, record=False):
    """SP method, Alg. 1: x_{k+1} = B x_k + c with P = Abar1^{-1}, B = P Abar2, c = P bbar.

    P is applied through a Cholesky factor of Abar1 (the same operator as the
    explicit inverse of Alg. 1 step 2).  Before each update the relative residual
    of the current iterate is compared with ``tol`` (Sec. 5 stops on the residual
    of x_k); ``outer_iters`` is the number of updates made.  ``b`` may hold k
    right-hand sides as columns; then every column runs to its own tolerance.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    G1, G2 = gram_blocks(A, p)
    L = np.linalg.cholesky(G1)
    bb = rhs_bar(A, b, p)
    B = _chol_solve(L, G2)
    c = _chol_solve(L, bb)
    multi = b.ndim == 2
    x = np.zeros_like(bb) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    info = SolveInfo()
    bnorm = np.linalg.norm(bb, axis=0)
    active = np.ones(bb.shape[1], dtype=bool) if multi else None
    iters = np.zeros(bb.shape[1], dtype=np.int64) if multi else 0
    for k in range(max_outer + 1):
        rel = np.linalg.norm(residual(A, b, p, x), axis=0) / bnorm
        info.history.append(rel)
        if record:
            info.iterates.append(x.copy())
        if multi:
            active = rel > tol
            if not active.any() or k == max_outer:
                break
            x[:, active] = B @ x[:, active] + c[:, active]
            iters[active] += 1
        else:
            if rel <= tol or k == max_outer:
                break
            x = B @ x + c
            iters += 1
    info.outer_iters = iters
    info.relres = rel
    info.converged = bool(np.all(rel <= tol))
    return x, info


def column_cumsum(A1):
    """Squared column norms ||A_1(:,j)||^2 and their running sum, added left to right.

    The running sum is the inverse-CDF table for the column distribution
    ||A_1(:,j)||^2 / ||A_1||_F^2 of Alg. 2 steps 8 and 10.
    """
    A1 = np.asarray(A1, dtype=np.float64)
    norms2 = np.einsum("ij,ij->j", A1, A1)
    cum = np.empty_like(norms2)
    s = 0.0
    for j in range(norms2.shape[0]):
        s += norms2[j]
        cum[j] = s
    return norms2, cum


def invcdf_pick(cum, u):
    """Column index for uniform u in [0,1): the smallest j with cum[j] > u * cum[-1]."""
    thr = u * cum[-1]
    j = int(np.searchsorted(cum, thr, side="right"))
    return min(j, cum.shape[0] - 1)


def scd_rank_from_uniform(u, n):
    """Rank i in 1..n with P(i) = (n+1) / (n i (i+1)), by inverse CDF.

    This is the law of the position, in decreasing order of |r|, of the index
    that Alg. 5 picks when alpha ~ U{1..n} and the subset is uniform (the
    reading of steps 7-9 taken here; see ``scd_rank_law``).  The CDF is
    (n+1)/n * i/(i+1), so i = ceil(u n / (n + 1 - u n)).
    """
    num = u * n
    i = math.ceil(num / ((n + 1) - num))
    return min(max(i, 1), n)


def scd_pick_rank(r, u):
    """Index of the i-th largest |r_s| (ties: lowest index), i from ``scd_rank_from_uniform``."""
    n = r.shape[0]
    i = scd_rank_from_uniform(u, n)
    order = np.lexsort((np.arange(n), -np.abs(r)))  # by decreasing |r|, then by index
    return int(order[i - 1])


def scd_pick_literal(r, alpha, subset):
    """Alg. 5 step 9: argmax over the subset of r_s^2, lowest index on ties."""
    best = None
    for s in sorted(int(v) for v in subset):
        if best is None or r[s] * r[s] > r[best] * r[best]:
            best = s
    return best


def scd_literal_law(absr):
    """Exact law of the picked index under alpha ~ U{1..n}, uniform alpha-subset.

    Enumerates every subset; for tiny n only.  ``absr`` must be tie-free.
    """
    from itertools import combinations
    n = len(absr)
    prob = np.zeros(n)
    for alpha in range(1, n + 1):
        subs = list(combinations(range(n), alpha))
        for tau in subs:
            j = max(tau, key=lambda s: (absr[s], -s))
            prob[j] += 1.0 / (n * len(subs))
    return prob


def scd_rank_law(absr):
    """Law of the picked index under the rank sampler (i-th largest with P(i) = (n+1)/(n i (i+1)))."""
    n = len(absr)
    order = sorted(range(n), key=lambda s: (-absr[s], s))
    prob = np.zeros(n)
    for i in range(1, n + 1):
        prob[order[i - 1]] = (n + 1) / (n * i * (i + 1))
    return prob


FIXED_ALPHA_SEARCH_MAX = 16  # alpha up to this: bisection on the first product form


def scd_fixed_survival(i, n, alpha):
    """P(rank > i) = C(n-i, alpha) / C(n, alpha) for a fixed subset size alpha (Sec. 4: a
    uniform alpha-subset, argmax of r_s^2 over it).

    The i-th largest |r_s| is picked exactly when it is in the subset and none of the i-1
    larger ones is, so the pick's rank exceeds i when the subset avoids the top i.
    Evaluated in FP64 as a product of exact-integer ratios, taken left to right:
      alpha <= FIXED_ALPHA_SEARCH_MAX:  prod_{s=0}^{alpha-1} (n-i-s) / (n-s)
      otherwise:                        prod_{s=0}^{i-1} (n-alpha-s) / (n-s)
    (both equal the binomial ratio; each is non-increasing in i after rounding, because
    every factor is, and a zero factor makes it 0 for i > n - alpha).
    """
    prod = 1.0
    if alpha <= FIXED_ALPHA_SEARCH_MAX:
        for s in range(alpha):
            num = n - i - s
            if num <= 0:
                return 0.0
            prod = prod * (float(num) / float(n - s))
    else:
        for s in range(i):
            num = n - alpha - s
            if num <= 0:
                return 0.0
            prod = prod * (float(num) / float(n - s))
    return prod


def scd_fixed_rank_from_uniform(u, n, alpha):
    """Rank i in 1..n-alpha+1 of the index picked with a fixed subset size alpha, by inverse
    CDF: the smallest i with P(rank > i) <= 1 - u (``scd_fixed_survival``).

    For small alpha the rank is found by bisection, otherwise by a scan from i = 1 (the
    expected rank is (n+1)/(alpha+1), small there).  alpha = n gives i = 1 (greedy, the
    Motzkin rule); alpha = 1 gives a uniform rank.
    """
    thr = 1.0 - u
    hi = n - alpha + 1
    if alpha <= FIXED_ALPHA_SEARCH_MAX:
        lo = 1
        while lo < hi:
            mid = (lo + hi) // 2
            if scd_fixed_survival(mid, n, alpha) <= thr:
                hi = mid
            else:
                lo = mid + 1
        return lo
    i = 1
    prod = float(n - alpha) / float(n)  # the survival at i = 1, extended one factor per step
    while i < hi and not (prod <= thr):
        prod = prod * (float(n - alpha - i) / float(n - i))
        i += 1
    return i


def scd_fixed_rank_law(absr, alpha):
    """Law of the picked index under the fixed-alpha rank sampler: the i-th largest |r_s|
    with probability C(n-i, alpha-1) / C(n, alpha)."""
    n = len(absr)
    order = sorted(range(n), key=lambda s: (-absr[s], s))
    prob = np.zeros(n)
    for i in range(1, n - alpha + 2):
        prob[order[i - 1]] = math.comb(n - i, alpha - 1) / math.comb(n, alpha)
    return prob


def scd_fixed_literal_law(absr, alpha):
    """Exact law of argmax over a uniform alpha-subset, by enumerating every subset (tiny n)."""
    from itertools import combinations
    n = len(absr)
    prob = np.zeros(n)
    subs = list(combinations(range(n), alpha))
    for tau in subs:
        j = max(tau, key=lambda s: (absr[s], -s))
        prob[j] += 1.0 / len(subs)
    return prob


def rk_step(A1, w, bhat, j, norms2):
    """RK step on A_1^T w = bhat (Alg. 2 step 9; RK of Sec. 3.1 on the rows of A_1^T).

    w + ((bhat_j - A_1(:,j)^T w) / ||A_1(:,j)||^2) A_1(:,j).
    """
    a = A1[:, j]
    return w + ((bhat[j] - a @ w) / norms2[j]) * a


def rgs_step(A1, z, w, j, norms2):
    """RGS step on A_1 z = w (Alg. 2 step 11; RGS of Sec. 3.2).

    z + (A_1(:,j)^T (w - A_1 z) / ||A_1(:,j)||^2) e_j, with A_1 z formed in full.
    """
    z = z.copy()
    z[j] += (A1[:, j] @ (w - A1 @ z)) / norms2[j]
    return z


def scd_step(G1, beta, r, j):
    """Coordinate step of Alg. 5 steps 10-11 on Abar1 beta = bhat, with r = bhat - Abar1 beta.

    delta = r_j / Abar1_jj; r - delta Abar1(:,j); beta + delta e_j.
    """
    delta = r[j] / G1[j, j]
    beta = beta.copy()
    beta[j] += delta
    return beta, r - delta * G1[:, j]


def theta_at(theta, k, theta_decay=1.0, theta_min=0.0):
    """Inner-stop factor of outer iteration k under a schedule (not in the paper, which
    leaves the inner stop open): theta_k = max(theta * theta_decay^k, theta_min).
    theta_decay = 1 (or <= 0) keeps theta constant."""
    if theta_decay <= 0.0 or theta_decay == 1.0:
        return theta
    return max(theta * theta_decay ** k, theta_min)


def sp_rk_rgs_solve(A, b, p, x0=None, tol=1e-12, max_outer=20000, max_inner=None, theta=0.1,
                    seed=0, chain=0, check_every=None, same_index=False, record=False, warm_inner=False,
                    theta_decay=1.0, theta_min=0.0):
    """SP-RK-RGS method, Alg. 2.

    Outer: bhat = Abar2 x_k + bbar (step 5), z = w = 0 (step 6).  Inner step t:
    draw j1 from the column distribution and take the RK step on A_1^T w = bhat
    (step 9); draw j2 and take the RGS step on A_1 z = w (step 11), using the
    updated w.  A_1 z is recomputed in full at every step (no maintained
    residual).  The inner loop stops after ``max_inner`` steps or once
    ||bhat - Abar1 z|| <= theta * ||bbar - H x_k||, tested every ``check_every``
    steps (the paper leaves the inner stop open).  x_{k+1} = z (step 13).

    Draws come from Philox4x32-10 (``step_uniforms(seed, chain, k, t)``): j1 from
    u0, j2 from u1, each by ``invcdf_pick``.  ``same_index`` forces j2 = j1,
    the SP-RCD special case of Sec. 4.

    ``warm_inner`` (not in the paper, which restarts at 0 in step 6) starts the inner
    solve at z = x_k, w = A_1 x_k instead: w stays in range(A_1), the inner fixed point
    Abar1^{-1} bhat is unchanged, and the start's residual bhat - Abar1 x_k is the outer
    residual bbar - H x_k, which the inner stop measures against.

    ``theta_decay`` / ``theta_min`` replace theta by ``theta_at(theta, k, ...)`` at outer
    iteration k (a schedule, not in the paper).
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    A1, A2 = A[:p], A[p:]
    G2 = A2.T @ A2  # step 2
    bb = rhs_bar(A, b, p)  # step 3
    norms2, cum = column_cumsum(A1)
    max_inner = 200 * n if max_inner is None else max_inner
    check_every = n if check_every is None else check_every
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(bb)
    info = SolveInfo()
    for k in range(max_outer + 1):
        r_out = residual(A, b, p, x)
        rel = np.linalg.norm(r_out) / bnorm
        info.history.append(rel)
        if record:
            info.iterates.append(x.copy())
        if rel <= tol or k == max_outer:
            break
        bhat = G2 @ x + bb
        w = A1 @ x if warm_inner else np.zeros(p)
        z = x.copy() if warm_inner else np.zeros(n)
        target = theta_at(theta, k, theta_decay, theta_min) * np.linalg.norm(r_out)
        t_done = max_inner
        for t in range(max_inner):
            u0, u1 = step_uniforms(seed, chain, k, t)
            j1 = invcdf_pick(cum, u0)
            w = rk_step(A1, w, bhat, j1, norms2)
            j2 = j1 if same_index else invcdf_pick(cum, u1)
            z = rgs_step(A1, z, w, j2, norms2)
            if record and k == 0:
                info.picks.append((j1, j2))
            if (t + 1) % check_every == 0:
                if np.linalg.norm(bhat - A1.T @ (A1 @ z)) <= target:
                    t_done = t + 1
                    break
        info.inner_iters.append(t_done)
        x = z
        info.outer_iters += 1
    info.relres = rel
    info.converged = rel <= tol
    return x, info


def sp_rk_rgs_gram_solve(A, b, p, x0=None, tol=1e-12, max_outer=20000, max_inner=None, theta=0.1,
                         seed=0, chain=0, check_every=None, same_index=False, warm_inner=False,
                         theta_decay=1.0, theta_min=0.0):
    """SP-RK-RGS, Alg. 2, with the inner vectors carried in Gram space (not in the paper).

    From w = 0, every RK step adds a multiple of a column of A_1 to w, so w = A_1 y for a
    coefficient vector y that gains delta in entry j1.  Keeping g = Abar1 y (= A_1^T w)
    and h = Abar1 z (= A_1^T A_1 z), the two steps of Alg. 2 become
        delta = (bhat_j1 - g_j1) / Abar1_{j1 j1};  y_j1 += delta;  g += delta Abar1(:, j1)
        eps   = (g_j2 - h_j2) / Abar1_{j2 j2};     z_j2 += eps;    h += eps Abar1(:, j2)
    because A_1(:,j)^T w = g_j, A_1(:,j)^T A_1 z = h_j and ||A_1(:,j)||^2 = Abar1_jj.  In
    exact arithmetic z is the iterate of the column form (``sp_rk_rgs_solve``) under the
    same draws, at O(n) work per step instead of O(p).  The inner stop reads
    ||bhat - h||, the exact quantity the column form recomputes.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    A1 = A[:p]
    G1, G2 = gram_blocks(A, p)
    bb = rhs_bar(A, b, p)
    norms2, cum = column_cumsum(A1)
    max_inner = 200 * n if max_inner is None else max_inner
    check_every = n if check_every is None else check_every
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(bb)
    info = SolveInfo()
    for k in range(max_outer + 1):
        r_out = residual(A, b, p, x)
        rel = np.linalg.norm(r_out) / bnorm
        info.history.append(rel)
        if rel <= tol or k == max_outer:
            break
        bhat = G2 @ x + bb
        z = x.copy() if warm_inner else np.zeros(n)
        g = G1 @ z  # w = A_1 z at a warm start (y = z), else w = 0
        h = g.copy()
        target = theta_at(theta, k, theta_decay, theta_min) * np.linalg.norm(r_out)
        t_done = max_inner
        for t in range(max_inner):
            u0, u1 = step_uniforms(seed, chain, k, t)
            j1 = invcdf_pick(cum, u0)
            delta = (bhat[j1] - g[j1]) / G1[j1, j1]
            g = g + delta * G1[:, j1]
            j2 = j1 if same_index else invcdf_pick(cum, u1)
            eps = (g[j2] - h[j2]) / G1[j2, j2]
            z = z.copy()
            z[j2] += eps
            h = h + eps * G1[:, j2]
            if (t + 1) % check_every == 0 and np.linalg.norm(bhat - h) <= target:
                t_done = t + 1
                break
        info.inner_iters.append(t_done)
        x = z
        info.outer_iters += 1
    info.relres = rel
    info.converged = rel <= tol
    return x, info


def sp_scd_solve(A, b, p, x0=None, tol=1e-12, max_outer=20000, max_inner=None, theta=0.1,
                 sampler="rank", alpha=None, seed=0, chain=0, record=False, rng=None, warm_inner=False,
                 theta_decay=1.0, theta_min=0.0):
    """SP-SCD method in the form the paper ran, Alg. 5.

    Outer: bhat = Abar2 x_k + bbar (step 4), beta = 0 and r = bhat (step 5).
    Inner step t: pick j (steps 7-9), then r -= (r_j / Abar1_jj) Abar1(:,j) and
    beta_j += r_j / Abar1_jj (steps 10-11, read with the current residual r_t).
    Before each inner step the loop stops if ||r|| <= theta * ||bbar - H x_k||,
    or after ``max_inner`` steps.  x_{k+1} = beta (step 13).

    Samplers for j:
      * ``"literal"``: alpha ~ U{1..n}, a uniform alpha-subset, argmax of r_s^2
        (ties to the lowest index); draws come from ``rng`` (numpy Generator).
      * ``"rank"``: the equal-in-law rank form, with the uniform u0 of
        ``step_uniforms(seed, chain, k, t)``.
      * ``"greedy"``: alpha = n, the Motzkin rule argmax_s r_s^2.
      * ``"fixed"``: a uniform subset of fixed size ``alpha`` (from ``rng``).
      * ``"fixed_rank"``: the equal-in-law rank form of ``"fixed"``: the i-th largest
        |r_s| with i = ``scd_fixed_rank_from_uniform(u0, n, alpha)``, u0 from Philox.

    ``warm_inner`` (not in the paper, which restarts at beta = 0 in step 5) starts the
    inner solve at beta = x_k, r = bhat - Abar1 x_k (= bbar - H x_k).  ``theta_decay`` /
    ``theta_min``: the schedule of ``theta_at``.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = A.shape[1]
    G1, G2 = gram_blocks(A, p)  # step 2
    bb = rhs_bar(A, b, p)
    max_inner = 200 * n if max_inner is None else max_inner
    if rng is None:
        rng = np.random.default_rng(seed)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(bb)
    info = SolveInfo()
    for k in range(max_outer + 1):
        r_out = residual(A, b, p, x)
        rel = np.linalg.norm(r_out) / bnorm
        info.history.append(rel)
        if record:
            info.iterates.append(x.copy())
        if rel <= tol or k == max_outer:
            break
        bhat = G2 @ x + bb
        beta = x.copy() if warm_inner else np.zeros(n)
        r = bhat - G1 @ beta
        target = theta_at(theta, k, theta_decay, theta_min) * np.linalg.norm(r_out)
        t_done = max_inner
        for t in range(max_inner):
            if np.linalg.norm(r) <= target:
                t_done = t
                break
            if sampler == "rank":
                u0, _ = step_uniforms(seed, chain, k, t)
                j = scd_pick_rank(r, u0)
            elif sampler == "greedy":
                j = scd_pick_literal(r, n, range(n))
            elif sampler == "literal":
                a_t = int(rng.integers(1, n + 1))
                j = scd_pick_literal(r, a_t, rng.choice(n, size=a_t, replace=False))
            elif sampler == "fixed":
                j = scd_pick_literal(r, alpha, rng.choice(n, size=alpha, replace=False))
            elif sampler == "fixed_rank":
                u0, _ = step_uniforms(seed, chain, k, t)
                i = scd_fixed_rank_from_uniform(u0, n, alpha)
                j = int(np.lexsort((np.arange(n), -np.abs(r)))[i - 1])
            else:
                raise ValueError(sampler)
            if record and k == 0:
                info.picks.append(j)
            beta, r = scd_step(G1, beta, r, j)
        info.inner_iters.append(t_done)
        x = beta
        info.outer_iters += 1
    info.relres = rel
    info.converged = rel <= tol
    return x, info
