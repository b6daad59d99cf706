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


def test_rayleigh_ritz_pins():
    """Rayleigh-Ritz on subspaces (the refinement step): full space = the
    closed form; a subspace holding the leading eigenvectors reproduces them;
    Ritz values are bounded by the eigenvalues and grow with the subspace
    (Courant-Fischer for the definite pencil (S_B, S_w + lambda I))."""
    P = lda_problem(3000, 24, 5, dtype="f64", seed=4)
    l, lam, k = 5, 1e-3, 4
    SB, Sw = L.scatters(P["X64"], P["y"], l)
    Swl = Sw + lam * np.eye(24)
    ref, Wref = L.lda_geneig(P["X64"], P["y"], l, lam, k)
    r_full, W_full = L.lda_rayleigh_ritz(SB, Swl, np.eye(24), k)
    assert np.allclose(r_full, ref, rtol=1e-10, atol=0)
    rng = np.random.default_rng(3)
    r_in, W_in = L.lda_rayleigh_ritz(SB, Swl, np.hstack([Wref, rng.standard_normal((24, 3))]), k)
    assert np.allclose(r_in, ref, rtol=1e-9, atol=0)
    assert np.allclose(W_in.T @ Swl @ W_in, np.eye(k), atol=1e-9)
    Wp = Wref + 0.05 * rng.standard_normal((24, k))
    eta = 0.05 * rng.standard_normal((24, k))
    r_k, _ = L.lda_rayleigh_ritz(SB, Swl, Wp, k)
    r_2k, _ = L.lda_rayleigh_ritz(SB, Swl, np.hstack([Wp, eta]), k)
    scale = ref[0]
    assert np.all(r_k <= ref + 1e-12 * scale) and np.all(r_2k <= ref + 1e-12 * scale)
    assert np.all(r_2k >= r_k - 1e-12 * scale)
    assert np.max(ref - r_2k) < np.max(ref - r_k)
