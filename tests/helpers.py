"""Shared test helpers: moving seeded inputs to the GPU in the C ABI's layouts."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def colmajor(A):
    """CUDA tensor (cols, rows) whose memory is the column-major rows x cols matrix A."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.float64).T)).to(dev())


def vec(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(dev())


def to_np_colmajor(t):
    """Back from a (cols, rows) CUDA tensor to a rows x cols numpy array."""
    return t.detach().cpu().numpy().T.copy()


def relerr(x, xs):
    return float(np.linalg.norm(np.asarray(x) - xs) / np.linalg.norm(xs))


def gemm_bound(X, Y, scale=4.0):
    """Elementwise FP64 error bound for X^T Y summed over K terms: scale * K * u * |X|^T |Y|."""
    K = X.shape[0]
    return scale * max(K, 1) * 2.0 ** -53 * (np.abs(X).T @ np.abs(Y))


def mlp_error_bounds(params, Theta, T, u_op=0.0, safety=1.0, lam=8.0):
    """First-order, entry-by-entry bounds on the FP32 errors of the warm-start network.

    Forward error analysis of each step of the GPU computation.  A dot product of length k
    contributes gamma_k |a|^T |b| with u = 2^-24 and the probabilistic constant
    gamma_k = lam sqrt(k) u of Higham & Mary (SIAM J. Sci. Comput. 41(5), 2019, Thm 3.1:
    it holds with probability >= 1 - 2k exp(-lam^2/2) under independent rounding errors;
    lam = 8 makes that 1e-11 per product; lam = None takes the worst case k u).  u_op is the rounding of the
    operands before each product, 2^-8 for BF16 inference, 0 for FP32; GELU and its
    derivative are charged 8 ulps of their arguments' scale), propagated through the
    layers with the exact FP64 activations of the oracle.  Returns (y_bound, grad_bound),
    both multiplied by `safety`.  grad_bound is flat, in the parameter layout.
    """
    import math
    from oracle import mlp as M

    W1, b1, W2, b2, W3, b3 = params
    u = 2.0 ** -24
    gam = (lambda k: k * u) if lam is None else (lambda k: lam * math.sqrt(k) * u)
    Th = np.asarray(Theta, dtype=np.float64)
    a = M.forward(params, Th)
    gp = lambda z: np.abs(M.gelu_grad(z))  # |g'|
    gpp = lambda z: np.abs(np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi) * (2.0 - z * z))  # |g''|

    def layer(h, e_h, W, b):
        k = W.shape[1] + 1
        aW, ah = np.abs(W), np.abs(h)
        return (gam(k) + 2 * u_op) * (ah @ aW.T + np.abs(b)) + e_h @ aW.T

    e_th = u_op * np.abs(Th)
    e_z1 = layer(Th, e_th, W1, b1)
    e_h1 = gp(a["z1"]) * e_z1 + 8 * u * np.abs(a["z1"]) + u_op * np.abs(a["h1"])
    e_z2 = layer(a["h1"], e_h1, W2, b2)
    e_h2 = gp(a["z2"]) * e_z2 + 8 * u * np.abs(a["z2"]) + u_op * np.abs(a["h2"])
    e_y = layer(a["h2"], e_h2, W3, b3)

    Tt = np.asarray(T, dtype=np.float64)
    B = Th.shape[0]
    count = a["y"].size
    diff = a["y"] - Tt
    e_dy = (2.0 / count) * (e_y + 2 * u * (np.abs(a["y"]) + np.abs(Tt)))
    dy = 2.0 * diff / count

    def back_w(d, e_d, h, e_hh):
        return gam(B) * (np.abs(d).T @ np.abs(h)) + e_d.T @ np.abs(h) + np.abs(d).T @ e_hh

    def back_b(d, e_d):
        return gam(B) * np.abs(d).sum(axis=0) + e_d.sum(axis=0)

    def back_act(d, e_d, W, z, e_z):
        k = W.shape[0]
        dh = d @ W
        e_dh = gam(k) * (np.abs(d) @ np.abs(W)) + e_d @ np.abs(W)
        e_dz = e_dh * gp(z) + np.abs(dh) * (gpp(z) * e_z + 8 * u * (gp(z) + 1.0)) + u * np.abs(dh * M.gelu_grad(z))
        return dh * M.gelu_grad(z), e_dz

    gW3, gb3 = back_w(dy, e_dy, a["h2"], e_h2), back_b(dy, e_dy)
    dz2, e_dz2 = back_act(dy, e_dy, W3, a["z2"], e_z2)
    gW2, gb2 = back_w(dz2, e_dz2, a["h1"], e_h1), back_b(dz2, e_dz2)
    dz1, e_dz1 = back_act(dz2, e_dz2, W2, a["z1"], e_z1)
    gW1, gb1 = back_w(dz1, e_dz1, Th, e_th), back_b(dz1, e_dz1)
    return safety * e_y, safety * M.flatten([gW1, gb1, gW2, gb2, gW3, gb3])
