"""Pins of the closed-form CCA oracle (Def. 4.1) against mathematics, not itself."""
import numpy as np
import pytest

from oracle import cca as C
from synth import cca_latent_problem


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def test_routes_agree_small(cfg_small):
    X, Y = cfg_small["X64"], cfg_small["Y64"]
    s1, U1, V1 = C.cca_whiten(X, Y, 1e-3, 1e-3, 5)
    s2, U2, V2 = C.cca_qr(X, Y, 1e-3, 1e-3, 5)
    assert _rel(s1, s2) < 1e-12
    assert np.max(np.abs(U1 - U2)) / np.max(np.abs(U2)) < 1e-8
    assert np.max(np.abs(V1 - V2)) / np.max(np.abs(V2)) < 1e-8


def test_constraints_and_critical_point(cfg_small):
    X, Y = cfg_small["X64"], cfg_small["Y64"]
    lam = 1e-3
    sig, U, V = C.cca_qr(X, Y, lam, lam, 5)
    Sxx, Syy, Sxy = C.sigmas(X, Y, lam, lam)
    I = np.eye(5)
    assert np.max(np.abs(U.T @ Sxx @ U - I)) < 1e-11
    assert np.max(np.abs(V.T @ Syy @ V - I)) < 1e-11
    assert np.max(np.abs(U.T @ Sxy @ V - np.diag(sig))) < 1e-11
    assert np.all(np.diff(sig) <= 0) and np.all(sig >= 0) and np.all(sig < 1)
    # critical-point equations of Thm 4.1 (App. B): Sxy V = Sxx U D, Sxy^T U = Syy V D
    assert np.max(np.abs(Sxy @ V - Sxx @ U @ np.diag(sig))) < 1e-8 * np.max(np.abs(Sxy @ V))
    assert np.max(np.abs(Sxy.T @ U - Syy @ V @ np.diag(sig))) < 1e-8 * np.max(np.abs(Sxy.T @ U))
    # objective at the optimum equals -sum sigma_i mu_i
    mu = C.default_mu(5)
    assert abs(C.cca_objective(U, V, Sxy, mu) + np.dot(sig, mu)) < 1e-11


def test_closed_form_identical_views():
    """X = Y, lambda > 0: sigma_i = s_i^2 / (s_i^2 + lambda), s_i singular values of X."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((200, 6)) @ np.diag([3, 2, 1, 0.5, 0.2, 0.05])
    lam = 0.01
    s = np.linalg.svd(X, compute_uv=False)
    expect = s ** 2 / (s ** 2 + lam)
    for fn in (C.cca_whiten, C.cca_qr, C.cca_geneig):
        sig, _, _ = fn(X, X, lam, lam, 6)
        assert _rel(sig, expect) < 1e-10


def test_brute_force_geneig_tiny():
    P = cca_latent_problem(30, 4, 3, latent=2, noise=0.7, seed=11)
    X, Y = P["X64"], P["Y64"]
    s1, U1, V1 = C.cca_geneig(X, Y, 0.1, 0.2, 3)
    s2, U2, V2 = C.cca_qr(X, Y, 0.1, 0.2, 3)
    s3, _, _ = C.cca_whiten(X, Y, 0.1, 0.2, 3)
    assert _rel(s1, s2) < 1e-10 and _rel(s3, s2) < 1e-10
    assert np.max(np.abs(U1 - U2)) < 1e-8 and np.max(np.abs(V1 - V2)) < 1e-8


def test_orthonormal_views_are_cosines():
    """lambda = 0 with orthonormal columns: sigma are the cosines of the
    principal angles between the column spaces (Sec. 4 intro)."""
    rng = np.random.default_rng(5)
    Qx, _ = np.linalg.qr(rng.standard_normal((50, 4)))
    Qy, _ = np.linalg.qr(rng.standard_normal((50, 3)))
    cosines = np.linalg.svd(Qx.T @ Qy, compute_uv=False)
    sig, _, _ = C.cca_qr(Qx, Qy, 0.0, 0.0, 3)
    assert _rel(sig, cosines) < 1e-12


def test_suboptimality_definition():
    sig = np.array([0.9, 0.5])
    mu = np.array([2.0, 1.0])
    assert C.suboptimality(sig, mu, -2.3) == pytest.approx(0.0)
    assert C.suboptimality(sig, mu, -2.0) == pytest.approx(0.3 / 2.3)


def test_rayleigh_ritz_pins(cfg_small):
    """Rayleigh-Ritz on subspaces (the refinement step): the whole space
    reproduces the closed form; a subspace holding the leading canonical
    weights (plus junk directions) reproduces them; any subspace gives Ritz
    values at most the canonical correlations, and a larger subspace that
    contains a smaller one gives values at least as large (Courant-Fischer for
    the pencil ([[0, Sxy], [Sxy^T, 0]], blkdiag(Sxx, Syy)))."""
    P = cfg_small
    lam, k = 1e-3, 5
    Sxx, Syy, Sxy = C.sigmas(P["X64"], P["Y64"], lam, lam)
    dx, dy = Sxy.shape
    ref, Uref, Vref = C.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    s_full, U_full, V_full = C.cca_rayleigh_ritz(Sxx, Syy, Sxy, np.eye(dx), np.eye(dy), k)
    assert np.allclose(s_full, ref, rtol=1e-10, atol=0)
    rng = np.random.default_rng(7)
    Bx = np.hstack([Uref, rng.standard_normal((dx, 3))])
    By = np.hstack([rng.standard_normal((dy, 2)), Vref])
    s_in, U_in, V_in = C.cca_rayleigh_ritz(Sxx, Syy, Sxy, Bx, By, k)
    assert np.allclose(s_in, ref, rtol=1e-10, atol=0)
    # the weights satisfy Def. 4.1's constraints
    assert np.allclose(U_in.T @ Sxx @ U_in, np.eye(k), atol=1e-9)
    assert np.allclose(U_in.T @ Sxy @ V_in, np.diag(s_in), atol=1e-9)
    # variational bound and monotonicity: U plus a perturbation direction
    Ux = Uref + 0.05 * rng.standard_normal((dx, k))
    Vy = Vref + 0.05 * rng.standard_normal((dy, k))
    ex = 0.05 * rng.standard_normal((dx, k))
    ey = 0.05 * rng.standard_normal((dy, k))
    s_k, _, _ = C.cca_rayleigh_ritz(Sxx, Syy, Sxy, Ux, Vy, k)
    s_2k, _, _ = C.cca_rayleigh_ritz(Sxx, Syy, Sxy, np.hstack([Ux, ex]), np.hstack([Vy, ey]), k)
    assert np.all(s_k <= ref + 1e-12) and np.all(s_2k <= ref + 1e-12)
    assert np.all(s_2k >= s_k - 1e-12)
    assert np.max(ref - s_2k) < np.max(ref - s_k)
