"""Helpers shared by the GPU parity tests (moving synthetic arrays to the device)."""
import numpy as np


def to_dev(a, dtype_name):
    import torch
    if dtype_name == "bf16":
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def np64(t):
    return t.detach().cpu().double().numpy()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def subspace_sin(U, V, B):
    """Largest sine of the principal angles between span(U) and span(V) in the B-inner product."""
    import scipy.linalg as sl
    L = np.linalg.cholesky(B)
    Qu, _ = np.linalg.qr(L.T @ U)
    Qv, _ = np.linalg.qr(L.T @ V)
    s = np.linalg.svd(Qu.T @ Qv, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - min(s) ** 2)))
