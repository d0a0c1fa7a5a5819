"""GPU parity of the warm-start network and of the warm-started solve.

* loss and gradients of the CUDA kernels against the FP64 oracle backprop (same FP32
  parameters), entry by entry, within the FP32 forward-error bound of each entry
  (``tests.helpers.mlp_error_bounds``);
* forward pass in FP32 and in BF16, entry by entry within the same kind of bound;
* the first Adam step against the oracle's update;
* on the warm-start configuration: a network trained on SP solutions predicts x0, the
  solve from x0 still meets ||x - x*|| / ||x*|| <= 1e-10, and takes fewer iterations
  than the solve from x0 = 0.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
import workloads as W
from tests.helpers import colmajor, mlp_error_bounds, relerr, to_np_colmajor

pytestmark = pytest.mark.gpu

D_IN, D_H, D_OUT = 16, 256, 256


@pytest.fixture(scope="module")
def ils():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2203_15340_gb300 as pkg
    return pkg


def tensors(theta, T):
    import torch
    th = torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float32)).cuda()
    Tt = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float64)).cuda()
    return th, Tt


def params_of(net):
    import torch
    p = torch.empty(net.num_params, dtype=torch.float32, device="cuda")
    net.get_params(p)
    torch.cuda.synchronize()
    return p.cpu().numpy().astype(np.float64)


def test_gradients_match_oracle_backprop(ils):
    import torch
    net = ils.WarmStartNet(D_IN, D_H, D_OUT, seed=11)
    rng = np.random.default_rng(3)
    theta = rng.uniform(-1, 1, size=(96, D_IN))
    T = rng.standard_normal((96, D_OUT)) * 0.5
    th, Tt = tensors(theta, T)
    grad = torch.empty(net.num_params, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(th, Tt, grad)
    flat = params_of(net)
    lo, go = M.loss_and_grad(M.unflatten(flat, D_IN, D_H, D_OUT), theta.astype(np.float32).astype(np.float64), T)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    g = grad.cpu().numpy().astype(np.float64)
    th64 = theta.astype(np.float32).astype(np.float64)
    _, gb = mlp_error_bounds(M.unflatten(flat, D_IN, D_H, D_OUT), th64, T)
    off = 0
    for shp in M.shapes(D_IN, D_H, D_OUT):
        size = int(np.prod(shp))
        err = np.abs(g[off:off + size] - go[off:off + size])
        bad = np.flatnonzero(err > gb[off:off + size])
        assert bad.size == 0, (shp, bad[:8], err[bad[:8]], gb[off:off + size][bad[:8]])
        off += size
    net.close()


def test_forward_fp32_and_bf16(ils):
    import torch
    net = ils.WarmStartNet(D_IN, D_H, D_OUT, seed=5)
    rng = np.random.default_rng(4)
    theta = rng.uniform(-1, 1, size=(300, D_IN))  # rows span 10 tiles of 32 and a ragged tail
    th, _ = tensors(theta, np.zeros((1, 1)))
    flat = params_of(net)
    params = M.unflatten(flat, D_IN, D_H, D_OUT)
    th64 = theta.astype(np.float32).astype(np.float64)
    yo = M.forward(params, th64)["y"]
    for bf16 in (False, True):
        yb, _ = mlp_error_bounds(params, th64, np.zeros_like(yo), u_op=2.0 ** -8 if bf16 else 0.0)
        X = torch.empty((300, D_OUT), dtype=torch.float64, device="cuda")
        net.forward(th, X, bf16=bf16)
        y = X.cpu().numpy()
        assert np.all(np.abs(y - yo) <= yb), (bf16, np.max(np.abs(y - yo) / yb))
    net.close()


def test_first_adam_step_matches_oracle(ils):
    import torch
    net = ils.WarmStartNet(D_IN, D_H, D_OUT, seed=7)
    rng = np.random.default_rng(8)
    theta = rng.uniform(-1, 1, size=(64, D_IN))
    T = rng.standard_normal((64, D_OUT)) * 2 + 1
    th, Tt = tensors(theta, T)
    p0 = params_of(net)
    lr = 1e-3
    net.train(th, Tt, epochs=1, batch=64, lr=lr)
    p1 = params_of(net)
    mu = T.mean(axis=0).astype(np.float32).astype(np.float64)
    sd = np.maximum(np.sqrt(np.maximum((T * T).mean(axis=0) - T.mean(axis=0) ** 2, 0)), 1e-12)
    sd = sd.astype(np.float32).astype(np.float64)
    Tn = ((T - mu) / sd).astype(np.float32).astype(np.float64)
    _, g = M.loss_and_grad(M.unflatten(p0, D_IN, D_H, D_OUT), theta.astype(np.float32).astype(np.float64), Tn)
    pe, _, _ = M.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, lr)
    big = np.abs(g) > 1e-4 * np.abs(g).max()  # away from g ~ eps, where the step flips
    assert np.allclose(p1[big], pe[big], rtol=0, atol=1e-3 * lr)
    net.close()


def warm_start_case(ils, n_train, n_eval, epochs):
    import torch
    fam = W.config5_warmstart()
    inst_A, p = fam.A, fam.p
    solver = ils.Solver(colmajor(inst_A), p, ils.options())
    th_train = fam.thetas(n_train, seed=5)
    th_eval = fam.thetas(n_eval, seed=55)
    B_train = fam.rhs(th_train, seed=5)
    B_eval = fam.rhs(th_eval, seed=55, start=0)
    # Targets: SP solutions produced by this library (Alg. 1 to relres 1e-12).
    X_train = torch.zeros((n_train, fam.A.shape[1]), dtype=torch.float64, device="cuda")
    for c0 in range(0, n_train, 2048):
        c1 = min(n_train, c0 + 2048)
        solver.solve_many(colmajor(B_train[:, c0:c1]), X_train[c0:c1], tol=1e-12)
    net = ils.WarmStartNet(16, 256, fam.A.shape[1], seed=1)
    th_t = torch.from_numpy(th_train.astype(np.float32)).cuda()
    loss = net.train(th_t, X_train, epochs=epochs, batch=256, lr=1e-3)
    th_e = torch.from_numpy(th_eval.astype(np.float32)).cuda()
    Be = colmajor(B_eval)
    X_cold = torch.zeros((n_eval, fam.A.shape[1]), dtype=torch.float64, device="cuda")
    X_warm = torch.zeros_like(X_cold)
    it_cold, it_warm = [], []
    for j in range(n_eval):
        ic = solver.solve_many(Be[j:j + 1], X_cold[j:j + 1], tol=1e-12)
        iw = net.solve(solver, th_e[j:j + 1], Be[j:j + 1], X_warm[j:j + 1], tol=1e-12)
        it_cold.append(ic.outer_iters)
        it_warm.append(iw.outer_iters)
    Xs = O.normal_equation_solve(fam.A, B_eval, p)
    errs = [relerr(to_np_colmajor(X_warm)[:, j], Xs[:, j]) for j in range(n_eval)]
    solver.close()
    net.close()
    return loss, np.mean(it_cold), np.mean(it_warm), max(errs)


def test_warm_start_saves_iterations_small(ils):
    loss, cold, warm, err = warm_start_case(ils, n_train=4096, n_eval=32, epochs=60)
    assert err <= 1e-10
    assert warm <= cold - 1.0, (cold, warm, loss)


def test_warm_start_full_configuration(ils):
    """50k SP solutions for training, 2k held-out parameters (seeds 5 / 55)."""
    loss, cold, warm, err = warm_start_case(ils, n_train=50000, n_eval=64, epochs=12)
    assert err <= 1e-10
    assert warm <= cold - 1.5, (cold, warm, loss)
