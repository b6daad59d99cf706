"""Generalized Stiefel manifold St_B(p, d) with a preconditioned metric (Table 1).

TEST INFRASTRUCTURE ONLY (see package docstring).

St_B(p, d) = {X in R^{d x p} : X^T B X = I_p} (Sec. 2), metric
g_X(xi, eta) = tr(xi^T M eta) for a fixed SPD M (Sec. 3 uses a constant M).
Every component below is the Table 1 formula written with dense B and M:

  normal projection    M^{-1} B X S, S the solution of the Sylvester equation
                       (X^T B M^{-1} B X) S + S (X^T B M^{-1} B X)
                           = X^T B xi + (X^T B xi)^T
  tangent projection   xi - M^{-1} B X S
  QR retraction        B^{-1/2} qf(B^{1/2} (X + xi)), qf = Q factor of the thin
                       QR with a positive diagonal R
  polar retraction     (X + xi)(I + xi^T B xi)^{-1/2}
  vector transport     projection of xi onto the tangent space at R_X(eta)
  Riemannian gradient  tangent projection of M^{-1} times the Euclidean gradient

``retr_chol`` is the same map as the QR retraction written with the Cholesky
factor of (X + xi)^T B (X + xi) (equal in exact arithmetic; a test checks it).

Parity: pinned by idempotence and self-adjointness of the projection, the
tangent-space equation, the closed form for M = B (xi - X sym(X^T B xi), used in
App. B's proof of Thm 4.1), agreement of the retraction forms, landing on the
manifold, and the directional-derivative identity
d/dt f(R_X(t eta))|_0 = g_X(grad f, eta) by finite differences
(tests/test_oracle_geometry.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def metric(M, xi, eta):
    return float(np.trace(xi.T @ M @ eta))


def sylvester_S(X, B, M, xi):
    BX = B @ X
    W = np.linalg.solve(M, BX)
    A = BX.T @ W
    C = BX.T @ xi
    S = sl.solve_sylvester(A, A, C + C.T)
    return S, W


def proj_normal(X, B, M, xi):
    S, W = sylvester_S(X, B, M, xi)
    return W @ S


def proj_tangent(X, B, M, xi):
    return xi - proj_normal(X, B, M, xi)


def _sqrt_pair(B):
    w, Q = np.linalg.eigh(B)
    return (Q * np.sqrt(w)) @ Q.T, (Q / np.sqrt(w)) @ Q.T


def retr_qr(X, B, xi):
    Bh, Bmh = _sqrt_pair(B)
    Q, R = np.linalg.qr(Bh @ (X + xi))
    Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    return Bmh @ Q


def retr_chol(X, B, xi):
    Y = X + xi
    L = np.linalg.cholesky(Y.T @ B @ Y)
    return sl.solve_triangular(L, Y.T, lower=True).T


def retr_polar(X, B, xi):
    p = X.shape[1]
    w, Q = np.linalg.eigh(np.eye(p) + xi.T @ B @ xi)
    return (X + xi) @ ((Q / np.sqrt(w)) @ Q.T)


def transport(X, B, M, eta, xi, retr=retr_qr):
    return proj_tangent(retr(X, B, eta), B, M, xi)


def rgrad(X, B, M, egrad):
    return proj_tangent(X, B, M, np.linalg.solve(M, egrad))


def on_manifold_error(X, B):
    return float(np.max(np.abs(X.T @ B @ X - np.eye(X.shape[1]))))
