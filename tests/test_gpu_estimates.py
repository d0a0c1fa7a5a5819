"""GPU checks of the Lanczos estimates, the stop rules, the TIMEOUT path and the attached
warm-start network.

* rho_est against the oracle's generalized eigensolve (Theorem 2.1's rho) and kappa_est
  against kappa_2(H) from the oracle's eigenvalues, within 1%, on every setup route
  (FP64 explicit, mixed overlapped, mixed with the FP64 factor, randomized); on the
  matrix-free route kappa_est is the bound kappa(Abar1) / (1 - rho), checked to lie above
  kappa_2(H);
* ILS_STOP_ERR_BOUND stops on kappa_est relres <= tol, so the returned x meets the
  oracle's x* to tol, and err_bound bounds the true error;
* Sec. 5's RR rule (relres^2 <= tol);
* an indefinite A^T J A on the matrix-free route is rejected at setup (rho_est >= 1);
* a grid-barrier wait bounded to 1 ns makes the one-launch solve return TIMEOUT, and the
  next solve on the same handle is correct.
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


@pytest.fixture(scope="module")
def c2():
    inst = W.config2()
    return inst, O.qr_cholesky_solve(inst.A, inst.b, inst.p), O.sp_spectral_radius(inst.A, inst.p), \
        O.normal_matrix_condition(inst.A, inst.p)


def solve(ils, inst, opts, tol, **kw):
    import torch
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(**opts))
    x = vec(np.zeros(inst.n))
    info = s.solve(vec(inst.b), x, tol=tol, **kw)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    s.close()
    return out, info


@pytest.mark.parametrize("opts", [
    dict(route=1),                              # FP64 SP, explicit route
    dict(precision=2),                          # mixed, overlapped setup (the headline path)
    dict(precision=1, factor64=1),              # mixed with the FP64 factorization
    dict(method=2),                             # SP-SCD: kappa only (P is never formed)
], ids=["fp64", "bf16_overlap", "fp32_factor64", "scd"])
def test_estimates_match_eigensolves(ils, c2, opts):
    inst, xs, rho, kap = c2
    x, info = solve(ils, inst, dict(estimate=1, **opts), tol=1e-12)
    assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
    assert abs(info.kappa_est - kap) <= 0.01 * kap, (info.kappa_est, kap)
    if opts.get("method", 0) == 0:
        assert abs(info.rho_est - rho) <= 0.01 * rho, (info.rho_est, rho)
    assert info.err_bound == pytest.approx(info.kappa_est * info.relres, rel=1e-12)
    assert info.err_bound >= relerr(x, xs)


def test_estimates_small_instance(ils):
    inst = W.config1()
    rho, kap = O.sp_spectral_radius(inst.A, inst.p), O.normal_matrix_condition(inst.A, inst.p)
    _, info = solve(ils, inst, dict(estimate=1), tol=1e-12)
    assert abs(info.kappa_est - kap) <= 0.01 * kap and abs(info.rho_est - rho) <= 0.01 * rho


def test_matrix_free_estimates_and_bound(ils):
    inst = W.dense_gaussian(2000, 4000, 48, 0.3, 21)  # q > 32 n: the matrix-free route
    rho, kap = O.sp_spectral_radius(inst.A, inst.p), O.normal_matrix_condition(inst.A, inst.p)
    xs = O.qr_cholesky_solve(inst.A, inst.b, inst.p)
    for prec in (0, 2):
        x, info = solve(ils, inst, dict(estimate=1, route=2, precision=prec), tol=1e-12)
        assert info.status == ils.ILS_OK and relerr(x, xs) <= 1e-10
        assert abs(info.rho_est - rho) <= 0.01 * rho, (prec, info.rho_est, rho)
        assert info.kappa_est >= 0.99 * kap, (prec, info.kappa_est, kap)  # kappa(Abar1) / (1 - rho) >= kappa(H)


def test_matrix_free_indefinite_rejected_at_setup(ils):
    bad = W.dense_gaussian(400, 1400, 40, 1.5, 5)
    assert not O.is_spd(O.normal_matrix(bad.A, bad.p)) and O.is_spd(bad.A[:bad.p].T @ bad.A[:bad.p])
    with pytest.raises(ils.ILSError) as e:
        ils.Solver(colmajor(bad.A), bad.p, ils.options(route=2, estimate=1))
    assert e.value.code == ils.ILS_ERR_NOT_SPD


@pytest.mark.parametrize("prec", [0, 2])
def test_error_bound_stop_rule(ils, c2, prec):
    """tol is the target relative error: the solve stops once kappa_est relres <= 1e-10."""
    inst, xs, _, kap = c2
    x, info = solve(ils, inst, dict(stop_rule=ils.ILS_STOP_ERR_BOUND, precision=prec), tol=1e-10)
    assert info.status == ils.ILS_OK
    assert info.err_bound <= 1e-10 and info.kappa_est * info.relres <= 1e-10
    assert relerr(x, xs) <= 1e-10 and relerr(x, xs) <= info.err_bound


def test_paper_rr_stop_rule(ils):
    """Sec. 5 stops when RR = relres^2 < 1e-6; the oracle's SP takes the same number of steps."""
    inst = W.config1()
    x, info = solve(ils, inst, dict(stop_rule=ils.ILS_STOP_PAPER_RR), tol=1e-6)
    assert info.status == ils.ILS_OK and info.relres ** 2 <= 1e-6
    _, oinfo = O.sp_solve(inst.A, inst.b, inst.p, tol=1e-3)
    assert info.outer_iters == oinfo.outer_iters
    assert O.paper_rr(inst.A, inst.b, inst.p, x) <= 1e-6 * (1 + 1e-6)


def test_timing_fields(ils):
    inst = W.config1()
    _, info = solve(ils, inst, dict(timing=1, method=2), tol=1e-12)
    assert info.t_solve_ms > 0 and info.t_setup_ms > 0 and info.t_inner_ms > 0


def test_timeout_then_next_solve_is_correct(ils, c2):
    """A 1 ns bound on the one-launch solve's grid-barrier waits cannot be met: the kernel
    records TIMEOUT, releases the other CTAs and returns; the handle stays usable."""
    import torch
    inst, xs, _, _ = c2
    s = ils.Solver(colmajor(inst.A), inst.p, ils.options(precision=ils.ILS_BF16_REFINE))
    x = vec(np.zeros(inst.n))
    s.set_wait_limit(1)
    info = s.solve(vec(inst.b), x, tol=1e-12, allow=(ils.ILS_ERR_TIMEOUT,))
    assert info.status == ils.ILS_ERR_TIMEOUT
    s.set_wait_limit(0)
    x.zero_()
    info = s.solve(vec(inst.b), x, tol=1e-12)
    torch.cuda.synchronize()
    assert info.status == ils.ILS_OK and relerr(x.cpu().numpy(), xs) <= 1e-10
    s.close()


def test_attached_warm_start_network(ils):
    """ils_set_warmstart + ils_solve_param(net = NULL) equals passing the network directly."""
    import torch
    fam = W.config5_warmstart()
    s = ils.Solver(colmajor(fam.A), fam.p, ils.options())
    net = ils.WarmStartNet(16, 256, fam.A.shape[1], seed=3)
    th = fam.thetas(4, seed=7)
    B = colmajor(fam.rhs(th, seed=7))
    tht = torch.from_numpy(th.astype(np.float32)).cuda()
    X1 = torch.zeros((4, fam.A.shape[1]), dtype=torch.float64, device="cuda")
    X2 = torch.zeros_like(X1)
    i1 = net.solve(s, tht, B, X1, tol=1e-12)
    s.set_warmstart(net)
    i2 = s.solve_param(tht, B, X2, tol=1e-12)
    torch.cuda.synchronize()
    assert i1.outer_iters == i2.outer_iters and torch.equal(X1, X2)
    s.set_warmstart(None)
    with pytest.raises(ils.ILSError):
        s.solve_param(tht, B, X2, tol=1e-12)
    net.close()
    s.close()
