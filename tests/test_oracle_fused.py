"""Pins of oracle.fused, the checker of the per-iteration data pass.

The pass products are pinned to the pinned covariance and scatter forms of
the closed-form oracles (oracle.cca.sigmas, Sec. 4.1 notation; oracle.lda.
scatters, Def. 5.1 / Sec. 5.1), and to a brute-force row-by-row loop on tiny
inputs.  A swapped pair of W blocks, a transposed operand or a dropped class
centring each fails one of these.
"""
import numpy as np
import pytest

from oracle import cca as OC
from oracle import fused as OF
from oracle import lda as OL
from synth import cca_latent_problem, lda_problem


def _phi(d, k2, seed):
    return np.random.default_rng(seed).standard_normal((d, k2))


def test_cca_pass_blocks_equal_covariance_products():
    """Gx = X^T [X Phi_x, Y Phi_y] = [(Sxx - lx I) Phi_x, Sxy Phi_y] and
    Gy = [Sxy^T Phi_x, (Syy - ly I) Phi_y]; the Gram of W is Phi_bd^T Sigma Phi_bd."""
    n, dx, dy, k2 = 700, 13, 9, 6
    P = cca_latent_problem(n, dx, dy, latent=4, dtype="f64", seed=3)
    X, Y = P["X64"], P["Y64"]
    lx, ly = 0.3, 0.7  # any value: the pass is independent of lambda
    Sxx, Syy, Sxy = OC.sigmas(X, Y, lx, ly)
    Px, Py = _phi(dx, k2, 1), _phi(dy, k2, 2)
    Gx, Gy, Gram = OF.cca_pass(X, Y, Px, Py)
    assert Gx.shape == (dx, 2 * k2) and Gy.shape == (dy, 2 * k2) and Gram.shape == (2 * k2, 2 * k2)
    sc = max(np.max(np.abs(Gx)), np.max(np.abs(Gy)))
    assert np.max(np.abs(Gx[:, :k2] - (Sxx - lx * np.eye(dx)) @ Px)) < 1e-12 * sc
    assert np.max(np.abs(Gx[:, k2:] - Sxy @ Py)) < 1e-12 * sc
    assert np.max(np.abs(Gy[:, :k2] - Sxy.T @ Px)) < 1e-12 * sc
    assert np.max(np.abs(Gy[:, k2:] - (Syy - ly * np.eye(dy)) @ Py)) < 1e-12 * sc
    Cxx = Px.T @ (Sxx - lx * np.eye(dx)) @ Px
    Cyy = Py.T @ (Syy - ly * np.eye(dy)) @ Py
    Cxy = Px.T @ Sxy @ Py
    exp = np.block([[Cxx, Cxy], [Cxy.T, Cyy]])
    assert np.max(np.abs(Gram - exp)) < 1e-12 * np.max(np.abs(exp))
    # the Gram is also Phi_bd^T G (how the library forms it from the pass)
    assert np.max(np.abs(Gram[:k2] - Px.T @ Gx)) < 1e-12 * np.max(np.abs(exp))
    assert np.max(np.abs(Gram[k2:] - Py.T @ Gy)) < 1e-12 * np.max(np.abs(exp))


def test_cca_pass_bruteforce_rows():
    """Tiny inputs: every entry summed row by row in plain Python loops."""
    n, dx, dy, k2 = 9, 3, 2, 2
    rng = np.random.default_rng(5)
    X, Y = rng.standard_normal((n, dx)), rng.standard_normal((n, dy))
    Px, Py = rng.standard_normal((dx, k2)), rng.standard_normal((dy, k2))
    Gx, Gy, Gram = OF.cca_pass(X, Y, Px, Py)
    for i_view, (Z, G) in enumerate(((X, Gx), (Y, Gy))):
        for j in range(Z.shape[1]):
            for c in range(2 * k2):
                s = 0.0
                for r in range(n):
                    if c < k2:
                        w = sum(X[r, a] * Px[a, c] for a in range(dx))
                    else:
                        w = sum(Y[r, a] * Py[a, c - k2] for a in range(dy))
                    s += Z[r, j] * w
                assert abs(G[j, c] - s) < 1e-12 * (1 + abs(s)), (i_view, j, c)
    for a in range(2 * k2):
        for b in range(2 * k2):
            s = 0.0
            for r in range(n):
                wa = sum(X[r, q] * Px[q, a] for q in range(dx)) if a < k2 else \
                    sum(Y[r, q] * Py[q, a - k2] for q in range(dy))
                wb = sum(X[r, q] * Px[q, b] for q in range(dx)) if b < k2 else \
                    sum(Y[r, q] * Py[q, b - k2] for q in range(dy))
                s += wa * wb
            assert abs(Gram[a, b] - s) < 1e-12 * (1 + abs(s))


def _swap_halves_cca_pass(X, Y, Px, Py):
    """A planted mistake: the two W blocks in the wrong order."""
    W = np.hstack([Y @ Py, X @ Px])
    return X.T @ W, Y.T @ W, W.T @ W


def test_planted_swap_is_caught():
    n, dx, dy, k2 = 300, 7, 7, 4
    P = cca_latent_problem(n, dx, dy, latent=3, dtype="f64", seed=4)
    X, Y = P["X64"], P["Y64"]
    Sxx, _, Sxy = OC.sigmas(X, Y, 0.0, 0.0)
    Px, Py = _phi(dx, k2, 1), _phi(dy, k2, 2)
    Gx, _, _ = _swap_halves_cca_pass(X, Y, Px, Py)
    sc = np.max(np.abs(Gx))
    assert np.max(np.abs(Gx[:, :k2] - Sxx @ Px)) > 1e-3 * sc


def test_lda_pass_equals_within_scatter_products():
    """Xhat^T (Xhat Phi) = S_w Phi and (Xhat Phi)^T (Xhat Phi) = Phi^T S_w Phi,
    S_w from the pinned scatter (Def. 5.1)."""
    n, d, l, k2 = 800, 11, 4, 6
    P = lda_problem(n, d, l, dtype="f64", seed=6)
    _, Sw = OL.scatters(P["X64"], P["y"], l)
    Phi = _phi(d, k2, 3)
    G, Gram = OF.lda_pass(P["X64"], P["y"], l, Phi)
    assert G.shape == (d, k2) and Gram.shape == (k2, k2)
    assert np.max(np.abs(G - Sw @ Phi)) < 1e-12 * np.max(np.abs(G))
    assert np.max(np.abs(Gram - Phi.T @ Sw @ Phi)) < 1e-12 * np.max(np.abs(Gram))


def test_lda_pass_class_centring_bruteforce():
    """Tiny inputs: centre each row by its class mean in loops, then sum."""
    n, d, l, k2 = 10, 3, 3, 2
    rng = np.random.default_rng(9)
    X = rng.standard_normal((n, d)) + 3.0
    y = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2, 2], dtype=np.int32)
    Phi = rng.standard_normal((d, k2))
    G, Gram = OF.lda_pass(X, y, l, Phi)
    means = []
    for c in range(l):
        rows = [r for r in range(n) if y[r] == c]
        means.append([sum(X[r, j] for r in rows) / len(rows) for j in range(d)])
    Xh = [[X[r, j] - means[y[r]][j] for j in range(d)] for r in range(n)]
    P = [[sum(Xh[r][j] * Phi[j, c] for j in range(d)) for c in range(k2)] for r in range(n)]
    for j in range(d):
        for c in range(k2):
            s = sum(Xh[r][j] * P[r][c] for r in range(n))
            assert abs(G[j, c] - s) < 1e-12 * (1 + abs(s))
    for a in range(k2):
        for b in range(k2):
            s = sum(P[r][a] * P[r][b] for r in range(n))
            assert abs(Gram[a, b] - s) < 1e-12 * (1 + abs(s))
    # without the centring the products differ (the class means are far from 0)
    Gu = X.T @ (X @ Phi)
    assert np.max(np.abs(Gu - G)) > 1e-2 * np.max(np.abs(G))


@pytest.mark.parametrize("view", [0, 1])
def test_cca_pass_linear_in_phi(view):
    """The pass is linear in each Phi block: doubling Phi_x doubles the first
    block column of Gx and Gy and leaves the second unchanged."""
    n, dx, dy, k2 = 200, 5, 4, 2
    P = cca_latent_problem(n, dx, dy, latent=2, dtype="f64", seed=7)
    Px, Py = _phi(dx, k2, 1), _phi(dy, k2, 2)
    a = OF.cca_pass(P["X64"], P["Y64"], Px, Py)
    b = OF.cca_pass(P["X64"], P["Y64"], 2 * Px, Py)
    G0, G1 = a[view], b[view]
    assert np.allclose(G1[:, :k2], 2 * G0[:, :k2], rtol=1e-13, atol=0)
    assert np.allclose(G1[:, k2:], G0[:, k2:], rtol=1e-13, atol=0)
