"""The seeded input recipes: determinism, shapes, scales and structure (CPU only).

These generators feed both the oracle and the CUDA path, so their recipe is checked on
its own: equal seeds give equal arrays, the shapes and the scales of A_1 and A_2 are the
stated ones, A^T J A is SPD where the recipe promises it, and the sparse pattern is valid
CSR.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _std(x):
    return float(np.std(x))


def test_dense_gaussian_is_deterministic_and_column_major():
    a = W.dense_gaussian(300, 80, 40, 0.3, 7)
    b = W.dense_gaussian(300, 80, 40, 0.3, 7)
    c = W.dense_gaussian(300, 80, 40, 0.3, 8)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.A, c.A)
    assert a.A.flags.f_contiguous and a.A.shape == (380, 40) and (a.p, a.q) == (300, 80)
    # b = A x_true + 1e-3 N(0, 1)
    r = a.b - a.A @ a.x_true
    assert 0.7e-3 < _std(r) < 1.3e-3


def test_dense_gaussian_many_rhs_blocks():
    inst = W.dense_gaussian(200, 50, 20, 0.3, 3, k=4)
    assert inst.b.shape == (250, 4) and inst.x_true.shape == (20, 4)
    assert inst.b.flags.f_contiguous
    r = inst.b - inst.A @ inst.x_true
    assert 0.7e-3 < _std(r) < 1.3e-3


@pytest.mark.parametrize("make,shape,p,a2", [(W.config1, (500, 50), 400, 0.2), (W.config2, (20000, 500), 16000, 0.3)])
def test_dense_configs_follow_their_recipe(make, shape, p, a2):
    inst = make()
    assert inst.A.shape == shape and inst.p == p and inst.q == shape[0] - p
    assert abs(_std(inst.A[:p]) - 1.0) < 0.02
    assert abs(_std(inst.A[p:]) / a2 - 1.0) < 0.02
    H = O.normal_matrix(inst.A, inst.p)
    assert O.is_spd(H)


def test_mp_scale_keeps_a_tall_a2_inside_the_spd_region():
    # the tall bandwidth case's scale, and the SPD margin it gives at a reduced size
    assert abs(W.mp_scale(16000, 262144, 500) - 0.0974) < 1e-3
    p, q, n = 2000, 32000, 100
    inst = W.dense_gaussian(p, q, n, W.mp_scale(p, q, n), 1)
    A1, A2 = inst.A[:p], inst.A[p:]
    lam_min_1 = np.linalg.eigvalsh(A1.T @ A1)[0]
    lam_max_2 = np.linalg.eigvalsh(A2.T @ A2)[-1]
    assert lam_max_2 < 0.5 * lam_min_1  # half the Marchenko-Pastur ratio, squared: about 1/4


def test_sparse_recipe_is_valid_csr_with_the_stated_law():
    m, n, p, dens = 2000, 60, 1600, 0.05
    s = W.config3_sparse(m=m, n=n, p=p, density=dens, seed=33)
    rp, ci, v = s.rowptr, s.colind, s.val
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and rp.shape == (m + 1,)
    assert rp[0] == 0 and rp[-1] == s.nnz and np.all(np.diff(rp) >= 0)
    assert np.all((ci >= 0) & (ci < n))
    for r in range(0, m, 97):  # strictly increasing columns within a row
        assert np.all(np.diff(ci[rp[r]:rp[r + 1]]) > 0)
    expect = m * n * dens
    assert abs(s.nnz - expect) < 5 * np.sqrt(expect)
    rows = np.repeat(np.arange(m), np.diff(rp))
    assert abs(_std(v[rows < p]) - 1.0) < 0.05
    assert abs(_std(v[rows >= p]) / 0.25 - 1.0) < 0.1
    D = np.zeros((m, n))
    D[rows, ci] = v
    r = s.b - D @ s.x_true
    assert 0.7e-3 < _std(r) < 1.3e-3


def test_batched_shapes_follow_the_recipe_and_the_matrices():
    shapes = W.config4_shapes()
    assert len(shapes) == 256
    for m, n, p, q in shapes:
        assert 32 <= n <= 512 and p + q == m
        assert 4.0 * n - 1 <= m <= 20.0 * n + 1
        assert 0.05 * m - 1 <= q <= 0.25 * m + 1
    assert len({n for _, n, _, _ in shapes}) > 100  # uneven sizes
    insts = W.config4_batched(count=256, k=2, indices=[0, 1, 255])
    for inst, i in zip(insts, [0, 1, 255]):
        assert (inst.m, inst.n, inst.p, inst.q) == shapes[i]
        assert inst.b.shape == (inst.m, 2)
        assert O.is_spd(O.normal_matrix(inst.A, inst.p))


def test_warm_start_rhs_slices_rebuild_exactly():
    fam = W.config5_warmstart(p=300, q=100, n=20, d=4)
    th = fam.thetas(10, 5)
    assert th.shape == (10, 4) and np.all(np.abs(th) <= 1.0)
    B = fam.rhs(th, 55)
    B2 = fam.rhs(th[6:], 55, start=6)
    assert np.array_equal(B[:, 6:], B2)
    r = B - fam.F @ th.T
    assert 0.7e-3 < _std(r) < 1.3e-3


def test_paper_table_shape():
    inst = W.paper_table_workload(300, 40, 30, diag=7.0)
    A1, A2 = inst.A[:300], inst.A[300:]
    assert np.all((A1 >= 0.0) & (A1 < 1.0))
    assert np.array_equal(A2, 7.0 * np.eye(40, 30))
    assert np.all((inst.b >= 0.0) & (inst.b < 1.0))
