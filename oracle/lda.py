"""Closed-form regularized Fisher LDA (Def. 5.1), two independent routes.

TEST INFRASTRUCTURE ONLY (see package docstring).

Def. 5.1: class means m_k, global mean m, between-class scatter
S_B = sum_k n_k (m_k - m)(m_k - m)^T, within-class scatter
S_w = sum_i (x_i - m_{y_i})(x_i - m_{y_i})^T.  The FDA weights are the leading
generalized eigenvectors of (S_B, S_w + lambda I) (Sec. 5.1), with eigenvalues
rho_1 >= rho_2 >= ... and at most l - 1 of them nonzero.  Sec. 5.1 factors
S_w = Xhat^T Xhat (row i of Xhat is x_i - m_{y_i}) and S_B = Yhat^T Yhat (row k
of Yhat is sqrt(n_k) (m_k - m)).

Routes
  lda_geneig  scipy.linalg.eigh(S_B, S_w + lambda I) on the explicit scatters.
  lda_qr      R from the QR of [Xhat; sqrt(lambda) I]; the rho are the squared
              singular values of Yhat R^{-1}.
  lda_rayleigh_ritz  the same problem restricted to a given subspace (the
              refinement step).

Parity: pinned by route agreement, the eigen-equation
S_B W = (S_w + lambda I) W diag(rho), W^T (S_w + lambda I) W = I, rank <= l - 1,
and the two-class closed form w ∝ (S_w + lambda I)^{-1} (m_1 - m_2)
(tests/test_oracle_lda.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl


def class_stats(X, y, l):
    X = np.asarray(X, dtype=np.float64)
    counts = np.bincount(y, minlength=l).astype(np.float64)
    sums = np.zeros((l, X.shape[1]))
    np.add.at(sums, y, X)
    means = sums / counts[:, None]
    m = X.mean(axis=0)
    Yhat = np.sqrt(counts)[:, None] * (means - m[None, :])
    Xhat = X - means[y]
    return counts, means, m, Yhat, Xhat


def scatters(X, y, l):
    _, _, _, Yhat, Xhat = class_stats(X, y, l)
    return Yhat.T @ Yhat, Xhat.T @ Xhat


def fix_signs(W):
    W = W.copy()
    for i in range(W.shape[1]):
        j = np.argmax(np.abs(W[:, i]))
        if W[j, i] < 0:
            W[:, i] *= -1
    return W


def lda_geneig(X, y, l, lam, k):
    SB, Sw = scatters(X, y, l)
    d = SB.shape[0]
    w, V = sl.eigh(SB, Sw + lam * np.eye(d))
    idx = np.argsort(w)[::-1][:k]
    return w[idx], fix_signs(V[:, idx])


def lda_qr(X, y, l, lam, k):
    _, _, _, Yhat, Xhat = class_stats(X, y, l)
    d = Xhat.shape[1]
    R = np.linalg.qr(np.vstack([Xhat, np.sqrt(lam) * np.eye(d)]), mode="r")
    R = np.where(np.diag(R) < 0, -1.0, 1.0)[:, None] * R
    G = sl.solve_triangular(R, Yhat.T, trans="T", lower=False).T  # Yhat R^{-1}
    _, s, Vt = np.linalg.svd(G, full_matrices=True)
    rho = np.zeros(d)
    rho[: s.shape[0]] = s ** 2
    W = sl.solve_triangular(R, Vt.T[:, :k], lower=False)
    return rho[:k], fix_signs(W)


def lda_rayleigh_ritz(SB, Swl, B, k):
    """Rayleigh-Ritz for Def. 5.1 on span(B): the generalized eigenproblem
    (B^T S_B B, B^T (S_w + lambda I) B) of the restricted problem, its leading
    k eigenpairs mapped back through B (the refinement step on W or on
    [W, eta]).  Swl = S_w + lambda I.  Pins: the full space gives lda_geneig;
    a subspace holding the leading eigenvectors gives them exactly; Ritz
    values never exceed the eigenvalues and do not decrease when the
    subspace grows (tests/test_oracle_lda.py)."""
    B = np.asarray(B, dtype=np.float64)
    w, V = sl.eigh(B.T @ SB @ B, B.T @ Swl @ B)
    idx = np.argsort(w)[::-1][:k]
    return w[idx], fix_signs(B @ V[:, idx])


def lda_objective(W, SB, mu):
    """f_FDA(W) = -1/2 tr(W^T S_B W N) (Sec. 5.2)."""
    return -0.5 * float(np.trace(W.T @ SB @ W @ np.diag(mu)))


def suboptimality(rho, mu, f):
    """Relative gap with the 1/2 of f_FDA carried into the optimum value:
    |1/2 sum rho_i mu_i + f| / (1/2 sum rho_i mu_i).  (Sec. 6.1 prints the CCA
    form without the 1/2, which would never vanish for f_FDA.)"""
    opt = 0.5 * float(np.dot(rho, mu))
    return abs(opt + f) / opt
