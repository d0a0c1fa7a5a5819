"""FP64 oracle of the warm-start network (test infrastructure only).

A three-layer perceptron theta -> x0 with GELU activations,
    z1 = W1 theta + b1, h1 = gelu(z1), z2 = W2 h1 + b2, h2 = gelu(z2), y = W3 h2 + b3,
its mean-squared-error loss against targets, the gradients by backpropagation, and one
Adam step (Kingma & Ba, "Adam: A method for stochastic optimization", ICLR 2015,
Algorithm 1).  gelu(z) = z Phi(z) with Phi the standard normal CDF (Hendrycks & Gimpel,
"Gaussian error linear units", 2016).

Parameters are stored flat, in the order W1 (h x d_in, row-major), b1, W2 (h x h), b2,
W3 (d_out x h), b3 -- the layout the CUDA library uses.  Only the tests may import this.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

__all__ = ["shapes", "unflatten", "flatten", "gelu", "gelu_grad", "forward", "loss_and_grad", "adam_step"]


def shapes(d_in, d_h, d_out):
    return [(d_h, d_in), (d_h,), (d_h, d_h), (d_h,), (d_out, d_h), (d_out,)]


def unflatten(flat, d_in, d_h, d_out):
    out, off = [], 0
    for shp in shapes(d_in, d_h, d_out):
        size = int(np.prod(shp))
        out.append(np.asarray(flat[off:off + size], dtype=np.float64).reshape(shp))
        off += size
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    Phi = 0.5 * (1.0 + erf(z / math.sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return Phi + z * phi


def forward(params, Theta):
    """Theta: (batch, d_in).  Returns the activations and the output y (batch, d_out)."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = Theta @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y}


def loss_and_grad(params, Theta, T):
    """loss = mean over all batch x d_out entries of (y - T)^2, and its gradient (flat)."""
    W1, b1, W2, b2, W3, b3 = params
    a = forward(params, Theta)
    diff = a["y"] - T
    count = diff.size
    loss = float(np.sum(diff * diff) / count)
    dy = 2.0 * diff / count
    gW3 = dy.T @ a["h2"]
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3
    dz2 = dh2 * gelu_grad(a["z2"])
    gW2 = dz2.T @ a["h1"]
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * gelu_grad(a["z1"])
    gW1 = dz1.T @ Theta
    gb1 = dz1.sum(axis=0)
    return loss, flatten([gW1, gb1, gW2, gb2, gW3, gb3])


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of flat arrays (t is the 1-based step count).  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
