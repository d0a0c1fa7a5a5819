"""GPU parity of mixed-precision SP with FP64 residual refinement.

Stated bounds: after refinement the FP32 and BF16 variants meet the same
||x - x*|| / ||x*|| <= 1e-10 as FP64 SP.  One correction step (three sweeps) must
contract the FP64 residual to at most 1e-3 (FP32 P and B) or 5e-2 (B in BF16) of its
start: rho(B)^3 plus the low-precision error of P and B times kappa(A^T J A).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import colmajor, relerr, to_np_colmajor, vec

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


def run(ils, inst, precision, tol=1e-12, **opt):
    import torch
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=precision, **opt))
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=tol, allow=(ils.ILS_OK, ils.ILS_ERR_NO_CONVERGENCE))
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    s.close()
    return out, info


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_mixed_reaches_fp64_accuracy(ils, prec, cfg):
    inst = W.config1() if cfg == "c1" else W.config2()
    precision = ils.ILS_FP32_REFINE if prec == "fp32" else ils.ILS_BF16_REFINE
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = run(ils, inst, precision, tol=1e-12)
    assert info.status == ils.ILS_OK
    assert relerr(x, xs) <= 1e-10
    assert 1 <= info.refinements <= (6 if prec == "fp32" else 12)
    assert info.relres <= 1e-12


@pytest.mark.parametrize("prec,bound", [("fp32", 1e-3), ("bf16", 5e-2)])
def test_one_correction_contracts_residual(ils, prec, bound):
    inst = W.config1()
    precision = ils.ILS_FP32_REFINE if prec == "fp32" else ils.ILS_BF16_REFINE
    x, info = run(ils, inst, precision, tol=0.0, max_outer=1)
    assert info.refinements == 1
    assert O.relres(inst.A, inst.b, inst.p, x) <= bound


def test_mixed_many_rhs(ils):
    import torch
    inst = W.dense_gaussian(900, 200, 70, 0.3, 17, k=11)
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE))
    X = torch.zeros((11, 70), dtype=torch.float64, device="cuda")
    info = s.solve_many(colmajor(inst.b), X, tol=1e-12)
    Xg = to_np_colmajor(X)
    Xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    for j in range(11):
        assert relerr(Xg[:, j], Xs[:, j]) <= 1e-10
    s.close()


def test_mixed_precision_needs_sp(ils):
    inst = W.config1()
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE, method=ils.ILS_SP_SCD))
    assert e.value.code == ils.ILS_ERR_INVALID_ARG


def test_sweep_autotuner_picks_a_shape_and_keeps_results(ils):
    """The first mixed setup of an n tunes the sweep shape; solving with the tuned shape gives
    the same answer as the oracle to 1e-10 (the shape does not change the arithmetic)."""
    import torch
    inst = W.dense_gaussian(2400, 600, 300, 0.3, 77)
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_BF16_REFINE))
    for k in (1, 8):
        for bf16 in (False, True):
            sh = ils.binding.tuned_shape(inst.n, k, bf16)
            assert sh is not None
            warps, blocks = sh
            assert warps in (1, 2, 4, 8) and blocks >= 1
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=1e-12)
    torch.cuda.synchronize()
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), xs) <= 1e-10
    s.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_setup_rejects_indefinite_h(ils, prec):
    """A_1^T A_1 is SPD but A^T J A is not: the mixed setup (whose FP32 test of H on a third
    stream fails and is confirmed in FP64) reports NOT_SPD."""
    bad = W.dense_gaussian(400, 300, 60, 2.0, 3)
    assert not O.is_spd(O.normal_matrix(bad.A, bad.p))
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(bad.A), bad.p, ils.options(precision=prec))
    assert e.value.code == ils.ILS_ERR_NOT_SPD


def test_mixed_setup_falls_back_to_fp64_factor(ils):
    """A column of A_1 scaled by 2^64 puts an entry of A_1^T A_1 beyond the FP32 range, so the
    FP32 inverse of A_1^T A_1 (and the FP32 test of H) fail although both matrices are SPD:
    the setup must take the FP64 factorization and succeed, with L the FP64 Cholesky factor."""
    import torch
    inst = W.dense_gaussian(300, 240, 40, 0.3, 11)
    A = inst.A.copy()
    A[: inst.p, 0] *= 2.0 ** 64
    G1 = A[: inst.p].T @ A[: inst.p]
    assert G1[0, 0] > np.finfo(np.float32).max and O.is_spd(O.normal_matrix(A, inst.p))
    s = ils.Solver(colmajor(A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE))
    out = torch.zeros((inst.n, inst.n), dtype=torch.float64, device="cuda")
    s.get_matrix(ils.MAT_CHOL, out)
    torch.cuda.synchronize()
    L = to_np_colmajor(out)
    Lx = np.linalg.cholesky(G1)
    assert np.max(np.abs(L - Lx) / np.abs(np.diag(Lx))[None, :]) <= 1e-12
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=1e-14)
    torch.cuda.synchronize()
    assert info.status == ils.ILS_OK and info.relres <= 1e-14
    s.close()
    # Column scaling is a congruence (D A^T J A D), so rho(B) and the refinement's contraction
    # are those of the unscaled problem, and every component of x converges like any other.
    # The 2-norm relres, though, is dominated by the scaled row (relres 1e-14 leaves about
    # 1e-10 in the unscaled components), so accuracy is pinned without the stop rule: eight
    # refinements (tol = 0 never stops earlier) reach the rounding level in every component.
    s = ils.Solver(colmajor(A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE, max_outer=8))
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=0.0, allow=(ils.ILS_ERR_NO_CONVERGENCE,))
    torch.cuda.synchronize()
    assert info.status == ils.ILS_ERR_NO_CONVERGENCE and info.refinements == 8
    assert relerr(x.cpu().numpy(), O.qr_cholesky_solve(A, inst.b, inst.p)) <= 1e-11
    s.close()


def test_mixed_get_matrix_forms_fp64_factor_on_demand(ils):
    """The mixed setup factors A_1^T A_1 in FP32; asking for L still returns the FP64 factor."""
    import torch
    inst = W.config1()
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_BF16_REFINE))
    out = torch.zeros((inst.n, inst.n), dtype=torch.float64, device="cuda")
    s.get_matrix(ils.MAT_CHOL, out)
    torch.cuda.synchronize()
    A1 = inst.A[: inst.p]
    Lx = np.linalg.cholesky(A1.T @ A1)
    assert np.max(np.abs(to_np_colmajor(out) - Lx)) <= 1e-10 * np.max(np.abs(Lx))
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=1e-12)
    torch.cuda.synchronize()
    assert info.status == ils.ILS_OK
    assert relerr(x.cpu().numpy(), O.qr_cholesky_solve(inst.A, inst.b, inst.p)) <= 1e-10
    s.close()


@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 64, 97, 700])
def test_mixed_sizes_around_panel_edges(ils, n):
    """The FP32 factorization of A_1^T A_1 runs in 32-column panels: sizes below, at and past
    a panel edge (and a size with many panels) must all refine to FP64 accuracy."""
    inst = W.dense_gaussian(max(4 * n, 8), max(n, 2), n, 0.3, 100 + n)
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = run(ils, inst, ils.ILS_FP32_REFINE, tol=1e-12)
    assert info.status == ils.ILS_OK
    assert relerr(x, xs) <= 1e-10
    assert info.refinements <= 6


def test_mixed_large_n_takes_wide_inverse_blocks(ils):
    """n = 1200: 32-wide tiles of the Gauss-Jordan inverse would have to share CTAs, so it
    sweeps 64-wide pivot blocks; the solve must still refine to FP64 accuracy."""
    inst = W.dense_gaussian(4800, 1200, 1200, 0.3, 120)
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = run(ils, inst, ils.ILS_FP32_REFINE, tol=1e-12)
    assert info.status == ils.ILS_OK
    assert relerr(x, xs) <= 1e-10


def test_mixed_wide_blocks_reject_indefinite_h(ils):
    """n = 1100 (64-wide inverse blocks) with A^T J A indefinite: the FP32 test of H on the
    third stream fails, the FP64 factorization confirms it, and the setup reports NOT_SPD."""
    bad = W.dense_gaussian(3300, 2200, 1100, 2.0, 5)
    assert not O.is_spd(O.normal_matrix(bad.A, bad.p))
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(bad.A), bad.p, ils.options(precision=ils.ILS_FP32_REFINE))
    assert e.value.code == ils.ILS_ERR_NOT_SPD


def test_mixed_largest_n_takes_cholesky_route(ils):
    """n = 2304 has more lower tiles than one cooperative wave of the inverse holds at
    either block size (152 SMs), so the setup factors A_1^T A_1 and H by Cholesky in FP32
    and forms P from the factor; the solve must still refine to FP64 accuracy."""
    inst = W.dense_gaussian(9216, 2304, 2304, 0.3, 121)
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    x, info = run(ils, inst, ils.ILS_FP32_REFINE, tol=1e-12)
    assert info.status == ils.ILS_OK
    assert relerr(x, xs) <= 1e-10


# ---------------------------------------------------------------------------------------
# Many right-hand sides (k >= 32): A^T J B and every residual b - H X as FP64-accurate split
# digit products on the tensor cores, FP32 sweeps; every column must meet 1e-10.
# ---------------------------------------------------------------------------------------

def wide_case(ils, inst, k, precision, x0=None, **opt):
    import torch
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=precision, **opt))
    X = torch.zeros((k, inst.n), dtype=torch.float64, device="cuda")
    if x0 is not None:
        X.copy_(torch.from_numpy(np.ascontiguousarray(x0.T)))
    info = s.solve_many(colmajor(inst.b), X, x0_zero=x0 is None, tol=1e-12)
    torch.cuda.synchronize()
    Xg = to_np_colmajor(X)
    s.close()
    return Xg, info


@pytest.mark.parametrize("precision", [1, 2])
def test_wide_mixed_ragged_tiles(ils, precision):
    inst = W.dense_gaussian(900, 200, 70, 0.3, 17, k=40)  # n and k below one 128-wide tile
    Xg, info = wide_case(ils, inst, 40, precision)
    Xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    assert info.status == ils.ILS_OK and info.relres <= 1e-12 and info.refinements >= 1
    assert max(relerr(Xg[:, j], Xs[:, j]) for j in range(40)) <= 1e-10


def test_wide_mixed_two_blocks_with_start(ils):
    """1100 right-hand sides (a full 1024-column block and a ragged one), n = 300 (three
    tiles, the last ragged), half of them started from a given x0."""
    k = 1100
    inst = W.dense_gaussian(2600, 400, 300, 0.3, 23, k=k)
    Xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    x0 = Xs + 0.05 * np.random.default_rng(2).standard_normal(Xs.shape)
    Xg, info = wide_case(ils, inst, k, ils.ILS_BF16_REFINE, x0=x0)
    assert info.status == ils.ILS_OK and info.relres <= 1e-12
    errs = [relerr(Xg[:, j], Xs[:, j]) for j in range(k)]
    assert max(errs) <= 1e-10, max(errs)


def test_wide_mixed_error_bound_rule(ils):
    """kappa_est relres <= 1e-10 for every column: every column's true error is below 1e-10."""
    inst = W.dense_gaussian(1800, 400, 150, 0.3, 29, k=64)
    Xg, info = wide_case(ils, inst, 64, ils.ILS_FP32_REFINE, stop_rule=2)
    Xs = O.normal_equation_solve(inst.A, inst.b, inst.p)
    assert info.status == ils.ILS_OK and info.err_bound <= 1e-10
    assert max(relerr(Xg[:, j], Xs[:, j]) for j in range(64)) <= info.err_bound


def test_wide_mixed_from_network_start(ils):
    """The combined form: mixed-precision refinement of 96 parametric right-hand sides from
    a trained network's x0 meets 1e-10 on every column and needs no more refinements than
    the cold start."""
    import torch
    fam = W.config5_warmstart()
    n = fam.A.shape[1]
    plain = ils.Solver(colmajor(fam.A), fam.p, ils.options())
    th_tr = fam.thetas(2048, seed=5)
    Xtr = torch.zeros((2048, n), dtype=torch.float64, device="cuda")
    plain.solve_many(colmajor(fam.rhs(th_tr, seed=5)), Xtr, tol=1e-12)
    net = ils.WarmStartNet(16, 256, n, seed=1)
    net.train(torch.from_numpy(th_tr.astype(np.float32)).cuda(), Xtr, epochs=40, batch=256, lr=1e-3)
    th = fam.thetas(96, seed=55)
    B = fam.rhs(th, seed=55)
    s = ils.Solver(colmajor(fam.A), fam.p, ils.options(precision=ils.ILS_BF16_REFINE))
    Xw = torch.zeros((96, n), dtype=torch.float64, device="cuda")
    Xc = torch.zeros_like(Xw)
    iw = net.solve(s, torch.from_numpy(th.astype(np.float32)).cuda(), colmajor(B), Xw, tol=1e-12)
    ic = s.solve_many(colmajor(B), Xc, tol=1e-12)
    torch.cuda.synchronize()
    Xs = O.normal_equation_solve(fam.A, B, fam.p)
    for X in (Xw, Xc):
        Xg = to_np_colmajor(X)
        assert max(relerr(Xg[:, j], Xs[:, j]) for j in range(96)) <= 1e-10
    assert iw.status == ils.ILS_OK and iw.refinements <= ic.refinements
    net.close()
    s.close()
    plain.close()


def test_tune_cache_file(ils, tmp_path):
    """options.tune_cache: the sweep shapes tuned at setup are written to the file (a header
    naming the GPU, then one line per tuned key), and the handle solves as before."""
    import torch
    path = tmp_path / "sweep_tune.txt"
    inst = W.dense_gaussian(1500, 300, 190, 0.3, 91)
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE, tune_cache=str(path)))
    lines = path.read_text().splitlines()
    assert lines[0].startswith("ils-sweep-tune-v1 ")
    keys = {tuple(int(v) for v in ln.split()[:3]) for ln in lines[1:]}
    assert ((190 + 31) // 32, 1, 0) in keys and ((190 + 31) // 32, 8, 0) in keys
    for ln in lines[1:]:
        nb, kc, bf, w, b = (int(v) for v in ln.split())
        assert w in (1, 2, 4, 8) and b >= 1
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=1e-12)
    torch.cuda.synchronize()
    assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), O.qr_cholesky_solve(inst.A, inst.b, inst.p)) <= 1e-10
    s.close()


def test_fp32_refinement_paths_agree(ils):
    """The one-cluster FP32 refinement sweeps with P and Abar2 (B d + P r = P (Abar2 d + r)) and
    leaves B to be formed after its kernels; a caller's wait limit selects the grid-barrier
    kernel, which reads B and has it formed first.  Both reach x*, and one correction of each
    contracts the residual alike."""
    import torch
    inst = W.config2()
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    At = colmajor(inst.A)  # read by the asynchronous setup: kept alive until its solve
    b = vec(inst.b)  # in place before each asynchronous setup, as the solve after it requires
    s = ils.Solver(At, inst.p, ils.options(precision=ils.ILS_FP32_REFINE))
    out = {}
    for name, limit in (("cluster", 0), ("grid", 10 ** 9)):
        s.set_wait_limit(limit)
        s.refactor_async(At)  # B again after the solve's kernels (or before the grid kernel)
        x = vec(np.zeros(inst.n))
        info = s.solve(b, x, tol=1e-12)
        torch.cuda.synchronize()
        assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), xs) <= 1e-10, name
        one = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_FP32_REFINE, max_outer=1))
        one.set_wait_limit(limit)
        x1 = vec(np.zeros(inst.n))
        one.solve(vec(inst.b), x1, tol=0.0, allow=(ils.ILS_ERR_NO_CONVERGENCE,))
        torch.cuda.synchronize()
        out[name] = O.relres(inst.A, inst.b, inst.p, x1.cpu().numpy())
        one.close()
    s.close()
    assert out["cluster"] <= 1e-3 and out["grid"] <= 1e-3
    assert 0.2 <= out["cluster"] / out["grid"] <= 5.0
