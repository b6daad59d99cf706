"""Pins of the closed-form Fisher LDA oracle (Def. 5.1)."""
import numpy as np

from oracle import lda as L
from synth import lda_problem


def _small(n=600, d=12, l=4, seed=1):
    P = lda_problem(n, d, l, dtype="f64", seed=seed)
    return P["X64"], P["y"], l


def test_total_scatter_identity():
    """S_w + S_B equals the total scatter sum_i (x_i - m)(x_i - m)^T."""
    X, y, l = _small()
    SB, Sw = L.scatters(X, y, l)
    Xc = X - X.mean(axis=0)
    assert np.max(np.abs(SB + Sw - Xc.T @ Xc)) < 1e-9 * np.max(np.abs(Xc.T @ Xc))


def test_routes_agree_and_eigen_equations():
    X, y, l = _small()
    lam = 1e-2
    r1, W1 = L.lda_geneig(X, y, l, lam, l - 1)
    r2, W2 = L.lda_qr(X, y, l, lam, l - 1)
    assert np.max(np.abs(r1 - r2) / r1) < 1e-10
    assert np.max(np.abs(W1 - W2)) / np.max(np.abs(W1)) < 1e-8
    SB, Sw = L.scatters(X, y, l)
    Swl = Sw + lam * np.eye(X.shape[1])
    assert np.max(np.abs(W1.T @ Swl @ W1 - np.eye(l - 1))) < 1e-10
    assert np.max(np.abs(SB @ W1 - Swl @ W1 @ np.diag(r1))) < 1e-9 * np.max(np.abs(SB @ W1))
    # rank(S_B) <= l - 1: the l-th generalized eigenvalue vanishes
    rall, _ = L.lda_geneig(X, y, l, lam, l)
    assert rall[-1] < 1e-10 * rall[0]
    mu = np.arange(l - 1, 0, -1, dtype=float)
    assert abs(L.lda_objective(W1, SB, mu) + 0.5 * np.dot(r1, mu)) < 1e-9 * np.dot(r1, mu)


def test_two_class_closed_form():
    """l = 2: rho_1 = (n1 n2 / n) D^T (S_w + lam I)^{-1} D and w ∝ (S_w + lam I)^{-1} D,
    D = m_1 - m_2 (Def. 5.1 footnote: S_B = (n1 n2 / n) D D^T)."""
    X, y, l = _small(n=301, d=7, l=2, seed=4)
    lam = 0.5
    counts, means, _, _, Xhat = L.class_stats(X, y, 2)
    Swl = Xhat.T @ Xhat + lam * np.eye(7)
    D = means[0] - means[1]
    z = np.linalg.solve(Swl, D)
    rho = counts[0] * counts[1] / counts.sum() * D @ z
    for fn in (L.lda_geneig, L.lda_qr):
        r, W = fn(X, y, 2, lam, 1)
        assert abs(r[0] - rho) < 1e-10 * rho
        w = W[:, 0]
        cos = abs(w @ z) / np.linalg.norm(w) / np.linalg.norm(z)
        assert abs(cos - 1) < 1e-12
