"""Sketch preconditioner M = Z^T S^T S Z + lambda I held as its factor R (Sec. 3).

TEST INFRASTRUCTURE ONLY (see package docstring).

Sec. 3: a QR factorization of the stacked (s + d) x d matrix [S Z; sqrt(lambda) I]
gives an upper-triangular R with R^T R = M, i.e. a Cholesky factor of M,
after which M^{-1} v costs two triangular solves.  Here the QR is LAPACK's
Householder QR (numpy.linalg.qr) and the signs are fixed so diag(R) > 0,
which makes R the unique Cholesky factor.

Parity: pinned by R^T R = (SZ)^T (SZ) + lambda I, triangularity and a positive
diagonal, and by agreement with the Cholesky factor of the explicit Gram
(tests/test_oracle_sketch.py).
"""
from __future__ import annotations

import numpy as np


def precond_R(SZ: np.ndarray, lam: float) -> np.ndarray:
    SZ = np.asarray(SZ, dtype=np.float64)
    d = SZ.shape[1]
    A = np.vstack([SZ, np.sqrt(lam) * np.eye(d)])
    R = np.linalg.qr(A, mode="r")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return sgn[:, None] * R


def apply_Minv(R: np.ndarray, V: np.ndarray) -> np.ndarray:
    """M^{-1} V = R^{-1} (R^{-T} V) by two triangular solves."""
    import scipy.linalg as sl
    W = sl.solve_triangular(R, V, trans="T", lower=False)
    return sl.solve_triangular(R, W, lower=False)
