"""Closed-form regularized CCA (Def. 4.1), three independent routes.

TEST INFRASTRUCTURE ONLY (see package docstring).

Def. 4.1: the (lambda_x, lambda_y)-canonical correlations sigma_1 >= ... and
weights U, V maximize tr(U^T X^T Y V) subject to U^T Sxx U = I,
V^T Syy V = I and U^T Sxy V diagonal, with Sxx = X^T X + lambda_x I,
Syy = Y^T Y + lambda_y I, Sxy = X^T Y (Sec. 4.1 notation).  There is no mean
centering: the definition is a linear-algebra one.

Routes
  cca_whiten    form Sxx, Syy, Sxy explicitly, Cholesky-whiten and take the
                SVD of Lx^{-1} Sxy Ly^{-T}; the singular values are the
                canonical correlations (link to the SVD of
                Sxx^{-1/2} Sxy Syy^{-1/2}, App. B proof of Thm 4.1).
  cca_qr        Bjorck-Golub style: Householder QR of [X; sqrt(lx) I] and
                [Y; sqrt(ly) I]; singular values of Qx1^T Qy1 (the n-row
                blocks), stable when Sxx is ill-conditioned.
  cca_geneig    brute force for tiny inputs: the positive generalized
                eigenvalues of ([[0, Sxy], [Sxy^T, 0]], blkdiag(Sxx, Syy)).
  cca_rayleigh_ritz  the same problem restricted to given subspaces (the
                refinement step).

Parity: pinned by mutual agreement of the routes, the constraints of
Def. 4.1, the critical-point equations Sxy V = Sxx U diag(sigma) and
Sxy^T U = Syy V diag(sigma) (App. B, proof of Thm 4.1), the closed form for
X = Y, and 0 <= sigma < 1 for lambda > 0 (tests/test_oracle_cca.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def sigmas(X, Y, lx, ly):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Sxx = X.T @ X + lx * np.eye(X.shape[1])
    Syy = Y.T @ Y + ly * np.eye(Y.shape[1])
    Sxy = X.T @ Y
    return Sxx, Syy, Sxy


def fix_signs(U, V, Sxy=None):
    """Column-sign convention (Thm 4.1 'same phase'): u_i^T Sxy v_i >= 0 and the
    largest-magnitude entry of u_i positive; flips u_i and v_i together."""
    U = U.copy()
    V = V.copy()
    for i in range(U.shape[1]):
        j = np.argmax(np.abs(U[:, i]))
        if U[j, i] < 0:
            U[:, i] *= -1
            V[:, i] *= -1
    if Sxy is not None:
        ph = np.einsum("ij,ij->j", U, Sxy @ V)
        V[:, ph < 0] *= -1
    return U, V


def cca_whiten(X, Y, lx, ly, k):
    Sxx, Syy, Sxy = sigmas(X, Y, lx, ly)
    Lx = np.linalg.cholesky(Sxx)
    Ly = np.linalg.cholesky(Syy)
    C = sl.solve_triangular(Lx, sl.solve_triangular(Ly, Sxy.T, lower=True).T, lower=True)
    A, s, Bt = np.linalg.svd(C)
    U = sl.solve_triangular(Lx.T, A[:, :k], lower=False)
    V = sl.solve_triangular(Ly.T, Bt.T[:, :k], lower=False)
    U, V = fix_signs(U, V, Sxy)
    return s[:k], U, V


def _qr_R(A, lam):
    d = A.shape[1]
    Q, R = np.linalg.qr(np.vstack([A, np.sqrt(lam) * np.eye(d)]))
    sg = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sg[None, :], sg[:, None] * R


def cca_qr(X, Y, lx, ly, k):
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    Qx, Rx = _qr_R(X, lx)
    Qy, Ry = _qr_R(Y, ly)
    C = Qx[:n].T @ Qy[:n]
    A, s, Bt = np.linalg.svd(C)
    U = sl.solve_triangular(Rx, A[:, :k], lower=False)
    V = sl.solve_triangular(Ry, Bt.T[:, :k], lower=False)
    U, V = fix_signs(U, V, X.T @ Y)
    return s[:k], U, V


def cca_geneig(X, Y, lx, ly, k):
    Sxx, Syy, Sxy = sigmas(X, Y, lx, ly)
    dx, dy = Sxy.shape
    A = np.zeros((dx + dy, dx + dy))
    A[:dx, dx:] = Sxy
    A[dx:, :dx] = Sxy.T
    B = sl.block_diag(Sxx, Syy)
    w, Z = sl.eigh(A, B)
    idx = np.argsort(w)[::-1][:k]
    Z = Z[:, idx] * np.sqrt(2.0)  # z^T B z = 1 splits evenly between the views
    U, V = fix_signs(Z[:dx], Z[dx:], Sxy)
    return w[idx], U, V


def cca_rayleigh_ritz(Sxx, Syy, Sxy, Bx, By, k):
    """Rayleigh-Ritz for Def. 4.1 on span(Bx) x span(By): the regularized CCA
    of the problem restricted to U = Bx A, V = By C.  Its matrices are the
    projected ones, Bx^T Sxx Bx, By^T Syy By and Bx^T Sxy By; whitening and an
    SVD (as in cca_whiten) give the Ritz values and the small weights, mapped
    back through Bx, By.  This is the refinement step a8 on the final point
    (Bx = U) or on the point and the last search direction (Bx = [U, eta]).
    Pins: the full space gives the closed form; a subspace that contains the
    leading canonical weights gives them exactly; every Ritz value is at
    most the corresponding canonical correlation, and enlarging the subspace
    raises none of the gaps (tests/test_oracle_cca.py)."""
    Bx = np.asarray(Bx, dtype=np.float64)
    By = np.asarray(By, dtype=np.float64)
    Gx = Bx.T @ Sxx @ Bx
    Gy = By.T @ Syy @ By
    Cxy = Bx.T @ Sxy @ By
    Lx = np.linalg.cholesky(Gx)
    Ly = np.linalg.cholesky(Gy)
    Cw = sl.solve_triangular(Lx, sl.solve_triangular(Ly, Cxy.T, lower=True).T, lower=True)
    A, s, Ct = np.linalg.svd(Cw)
    U = Bx @ sl.solve_triangular(Lx.T, A[:, :k], lower=False)
    V = By @ sl.solve_triangular(Ly.T, Ct.T[:, :k], lower=False)
    U, V = fix_signs(U, V, Sxy)
    return s[:k], U, V


def cca_objective(U, V, Sxy, mu):
    """f_CCA(U, V) = -tr(U^T Sxy V N), N = diag(mu) (Sec. 4.2)."""
    return -float(np.trace(U.T @ Sxy @ V @ np.diag(mu)))


def suboptimality(sig, mu, f):
    """|sum sigma_i mu_i + f| / sum sigma_i mu_i (Sec. 6.1)."""
    opt = float(np.dot(sig, mu))
    return abs(opt + f) / opt


def default_mu(k):
    """Descending weights mu_i = k - i + 1 (reading of Sec. 6.1: descending
    integers; diag(3, 2.75, 2) is the paper's own choice for p = 3)."""
    return np.arange(k, 0, -1, dtype=np.float64)
