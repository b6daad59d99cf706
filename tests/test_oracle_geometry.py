"""Pins of the Table 1 geometry oracle by identities that hold for the exact maps."""
import numpy as np
import pytest

from oracle import geometry as G
from oracle.cca import sigmas, cca_qr, default_mu
from oracle.problems import CCAProblem, FDAProblem
from oracle.lda import scatters, lda_geneig
from synth import cca_latent_problem, lda_problem


def _spd(d, rng, cond=100.0):
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    return (Q * np.geomspace(1, cond, d)) @ Q.T


def _point(d, p, B, rng):
    return G.retr_chol(rng.standard_normal((d, p)), B, np.zeros((d, p)))


@pytest.fixture
def setup():
    rng = np.random.default_rng(0)
    d, p = 9, 3
    B = _spd(d, rng, 50.0)
    M = _spd(d, rng, 20.0)
    X = _point(d, p, B, rng)
    return rng, d, p, B, M, X


def test_projection_identities(setup):
    rng, d, p, B, M, X = setup
    xi = rng.standard_normal((d, p))
    eta = rng.standard_normal((d, p))
    P1 = G.proj_tangent(X, B, M, xi)
    # tangent-space equation: Z^T B X + X^T B Z = 0
    T = P1.T @ B @ X
    assert np.max(np.abs(T + T.T)) < 1e-11
    assert np.max(np.abs(G.proj_tangent(X, B, M, P1) - P1)) < 1e-11  # idempotent
    P2 = G.proj_tangent(X, B, M, eta)
    # self-adjoint in g, and the normal part is g-orthogonal to the tangent space
    assert abs(G.metric(M, P1, eta) - G.metric(M, xi, P2)) < 1e-10
    assert abs(G.metric(M, xi - P1, P2)) < 1e-10


def test_projection_standard_metric_closed_form(setup):
    """M = B: Pi(xi) = xi - X sym(X^T B xi) (App. B, proof of Thm 4.1)."""
    rng, d, p, B, M, X = setup
    xi = rng.standard_normal((d, p))
    A = X.T @ B @ xi
    assert np.max(np.abs(G.proj_tangent(X, B, B, xi) - (xi - X @ (A + A.T) / 2))) < 1e-11


def test_retractions(setup):
    rng, d, p, B, M, X = setup
    xi = G.proj_tangent(X, B, M, rng.standard_normal((d, p)))
    Rq = G.retr_qr(X, B, xi)
    assert np.max(np.abs(Rq - G.retr_chol(X, B, xi))) < 1e-10
    for r in (Rq, G.retr_polar(X, B, xi)):
        assert G.on_manifold_error(r, B) < 1e-11
    # first-order agreement with X + t xi
    for t in (1e-3, 1e-4):
        e = np.max(np.abs(G.retr_qr(X, B, t * xi) - X - t * xi))
        assert e < 50 * t * t * np.max(np.abs(xi)) ** 2 + 1e-13
    Tv = G.transport(X, B, M, xi, rng.standard_normal((d, p)))
    Y = G.retr_qr(X, B, xi)
    S = Tv.T @ B @ Y
    assert np.max(np.abs(S + S.T)) < 1e-10


def _fd_check(problem, Ms, pts, rng):
    eg = problem.egrad(pts)
    grads = [G.rgrad(x, B, M, g) for x, B, M, g in zip(pts, problem.Bs, Ms, eg)]
    etas = [G.proj_tangent(x, B, M, rng.standard_normal(x.shape)) for x, B, M in zip(pts, problem.Bs, Ms)]
    h = 1e-5
    fp = problem.cost([G.retr_qr(x, B, h * e) for x, B, e in zip(pts, problem.Bs, etas)])
    fm = problem.cost([G.retr_qr(x, B, -h * e) for x, B, e in zip(pts, problem.Bs, etas)])
    fd = (fp - fm) / (2 * h)
    an = sum(G.metric(M, g, e) for M, g, e in zip(Ms, grads, etas))
    return fd, an


def test_cca_gradient_directional_derivative():
    rng = np.random.default_rng(1)
    P = cca_latent_problem(80, 6, 5, latent=3, seed=2)
    Sxx, Syy, Sxy = sigmas(P["X64"], P["Y64"], 0.1, 0.1)
    prob = CCAProblem(Sxx, Syy, Sxy, default_mu(3))
    Ms = [_spd(6, rng, 10), _spd(5, rng, 10)]
    pts = [_point(6, 3, Sxx, rng), _point(5, 3, Syy, rng)]
    fd, an = _fd_check(prob, Ms, pts, rng)
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_fda_gradient_directional_derivative():
    rng = np.random.default_rng(2)
    P = lda_problem(200, 6, 4, dtype="f64", seed=3)
    SB, Sw = scatters(P["X64"], P["y"], 4)
    Swl = Sw + 0.1 * np.eye(6)
    prob = FDAProblem(SB, Swl, np.array([3.0, 2.0, 1.0]))
    Ms = [_spd(6, rng, 10)]
    fd, an = _fd_check(prob, Ms, [_point(6, 3, Swl, rng)], rng)
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_gradient_vanishes_at_closed_form_optimum():
    rng = np.random.default_rng(3)
    P = cca_latent_problem(120, 7, 6, latent=4, seed=4)
    Sxx, Syy, Sxy = sigmas(P["X64"], P["Y64"], 0.05, 0.05)
    _, U, V = cca_qr(P["X64"], P["Y64"], 0.05, 0.05, 3)
    prob = CCAProblem(Sxx, Syy, Sxy, default_mu(3))
    Ms = [_spd(7, rng, 30), _spd(6, rng, 30)]
    eg = prob.egrad([U, V])
    for x, B, M, g in zip([U, V], prob.Bs, Ms, eg):
        assert np.max(np.abs(G.rgrad(x, B, M, g))) < 1e-9 * np.max(np.abs(np.linalg.solve(M, g)))
    SB, Sw = scatters(lda_problem(150, 5, 3, dtype="f64", seed=5)["X64"],
                      lda_problem(150, 5, 3, dtype="f64", seed=5)["y"], 3)
