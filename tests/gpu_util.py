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


def bound_ratio(got, exp, ref, gamma):
    """Largest |got - exp| / (gamma * ref) over all entries: <= 1 means every
    entry is within its own error bound, ref being the entry's magnitude
    reference (the sum of |terms| that a rounding analysis bounds against)."""
    err = np.abs(np.asarray(got) - np.asarray(exp))
    lim = gamma * np.asarray(ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(err == 0, 0.0, err / np.where(lim > 0, lim, 1e-300))
    return float(np.max(r))


def cca_pass_refs(X, Y, Px, Py):
    """Magnitude references of the CCA pass outputs: with |W| <= [|X||Px|,
    |Y||Py|] entrywise, Gx = X^T W is bounded by |X|^T |W|, Gy likewise, and
    Gram = Phi_bd^T G by |Phi_bd|^T |G|-references."""
    aW = np.hstack([np.abs(X) @ np.abs(Px), np.abs(Y) @ np.abs(Py)])
    rx = np.abs(X).T @ aW
    ry = np.abs(Y).T @ aW
    rg = np.vstack([np.abs(Px).T @ rx, np.abs(Py).T @ ry])
    return rx, ry, rg, aW
