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
