"""Pins for the warm-start network's FP64 oracle: central finite differences of the loss,
the GELU derivative against its definition, and Adam's first step (CPU only)."""
import math

import numpy as np
from scipy.stats import norm

from oracle import mlp as M


def small_net(seed, d_in=3, d_h=5, d_out=4):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(sum(int(np.prod(s)) for s in M.shapes(d_in, d_h, d_out))) * 0.5
    return flat, (d_in, d_h, d_out)


def test_gelu_is_z_times_normal_cdf():
    z = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(z), z * norm.cdf(z), atol=1e-15)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


def test_backprop_matches_central_differences():
    flat, dims = small_net(0)
    rng = np.random.default_rng(1)
    Theta = rng.uniform(-1, 1, size=(7, dims[0]))
    T = rng.standard_normal((7, dims[2]))
    loss, g = M.loss_and_grad(M.unflatten(flat, *dims), Theta, T)
    h = 1e-6
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = M.loss_and_grad(M.unflatten(flat + e, *dims), Theta, T)
        lm, _ = M.loss_and_grad(M.unflatten(flat - e, *dims), Theta, T)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-7 * (1 + abs(g[i])), i


def test_forward_shapes_and_linear_limit():
    """With W1, W2 tiny the hidden layers are near-linear around 0: gelu(z) ~ z/2."""
    d_in, d_h, d_out = 4, 6, 3
    rng = np.random.default_rng(2)
    W1 = rng.standard_normal((d_h, d_in)) * 1e-4
    W2 = rng.standard_normal((d_h, d_h))
    W3 = rng.standard_normal((d_out, d_h))
    params = [W1, np.zeros(d_h), W2, np.zeros(d_h), W3, np.zeros(d_out)]
    Theta = rng.uniform(-1, 1, size=(5, d_in))
    y = M.forward(params, Theta)["y"]
    approx = (0.5 * (0.5 * (Theta @ W1.T)) @ W2.T) @ W3.T
    assert y.shape == (5, d_out)
    assert np.allclose(y, approx, rtol=1e-3, atol=1e-9)


def test_adam_first_step_is_signed_lr():
    """At t = 1 the bias-corrected Adam step is lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def _fp32_network_sim(params, Theta, T):
    """The network's loss gradient evaluated entirely in numpy float32 (a stand-in for an
    FP32 device computation; only the bound helper is under test here)."""
    from scipy.special import erf
    f = np.float32
    W1, b1, W2, b2, W3, b3 = [p.astype(f) for p in params]
    th = Theta.astype(f)

    def gelu(z):
        return (f(0.5) * z * (f(1) + erf(z * f(0.70710678)).astype(f))).astype(f)

    def gelu_grad(z):
        Phi = (f(0.5) * (f(1) + erf(z * f(0.70710678)).astype(f))).astype(f)
        return (Phi + z * (np.exp(-f(0.5) * z * z) / f(math.sqrt(2 * math.pi))).astype(f)).astype(f)

    z1 = th @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    dy = (f(2) * (y - T.astype(f)) / f(y.size)).astype(f)
    dz2 = (dy @ W3) * gelu_grad(z2)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    return y, M.flatten([dz1.T @ th, dz1.sum(0), dz2.T @ h1, dz2.sum(0), dy.T @ h2, dy.sum(0)])


def test_fp32_error_bounds_hold_and_catch_wrong_entries():
    """The entry-by-entry bounds the GPU gradient test uses: an FP32 evaluation stays inside
    them, while one entry off by 1e-3 relative, swapped with its neighbour or zeroed falls
    outside."""
    from tests.helpers import mlp_error_bounds
    d_in, d_h, d_out = 16, 64, 48
    rng = np.random.default_rng(12)
    params = []
    for shp in M.shapes(d_in, d_h, d_out):
        fan = shp[1] if len(shp) == 2 else d_in
        params.append((rng.uniform(-1, 1, size=shp) / math.sqrt(fan)).astype(np.float32).astype(np.float64))
    Theta = rng.uniform(-1, 1, size=(40, d_in)).astype(np.float32).astype(np.float64)
    T = rng.standard_normal((40, d_out))
    _, go = M.loss_and_grad(params, Theta, T)
    yo = M.forward(params, Theta)["y"]
    y32, g32 = _fp32_network_sim(params, Theta, T)
    yb, gb = mlp_error_bounds(params, Theta, T)
    assert np.all(np.abs(g32 - go) <= gb) and np.all(np.abs(y32 - yo) <= yb)
    i = int(np.argmax(np.abs(go)))
    for bad in (g32 * np.where(np.arange(g32.size) == i, 1.001, 1.0),
                np.where(np.arange(g32.size) == i, 0.0, g32),
                np.where(np.arange(g32.size) == i, g32[i + 1], g32)):
        assert np.any(np.abs(bad - go) > gb)
