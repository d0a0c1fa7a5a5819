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
