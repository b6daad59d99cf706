"""Pins of the reference Riemannian CG and Algorithms 1-2 in the oracle."""
import numpy as np

from oracle import rcg as RC
from oracle.cca import sigmas, cca_qr, default_mu, suboptimality
from oracle.lda import scatters, lda_geneig, class_stats
from oracle.problems import CCAProblem, FDAProblem
from oracle import rng as R
from oracle.sketch import countsketch_apply
from synth import cca_latent_problem, lda_problem


def test_algorithm1_small_fp64(cfg_small):
    """Alg. 1 on the plain FP64 workload converges to the closed form."""
    X, Y = cfg_small["X64"], cfg_small["Y64"]
    lam, k, s = 1e-3, 5, 360
    h, g = R.countsketch_hash(2000, s, seed=0)
    SX, SY = countsketch_apply(X, h, g, s), countsketch_apply(Y, h, g, s)
    mu = default_mu(k)
    # the leading correlations are all ~0.99 with gaps ~3e-4, so the Riemannian
    # Hessian is ill-conditioned (Thm 4.4) and CG needs a few thousand steps
    res = RC.cca_algorithm1(X, Y, lam, lam, k, mu, SX, SY, gtol=1e-10, max_iter=6000)
    sig, _, _ = cca_qr(X, Y, lam, lam, k)
    assert res["status"] in ("converged", "stalled")
    assert np.max(np.abs(res["sigma"] - sig) / sig) < 1e-9
    assert suboptimality(sig, mu, res["f"]) < 1e-11


def test_rgd_p1_is_als():
    """Sec. 6.2: RGD with the standard metric and step 1/(u^T Sxy v) is ALS."""
    P = cca_latent_problem(150, 6, 5, latent=3, seed=8)
    Sxx, Syy, Sxy = sigmas(P["X64"], P["Y64"], 0.1, 0.1)
    rng = np.random.default_rng(0)
    u0, v0 = rng.standard_normal((6, 1)), rng.standard_normal((5, 1))
    if (u0.T @ Sxy @ v0).item() < 0:
        v0 = -v0
    prob = CCAProblem(Sxx, Syy, Sxy, np.array([1.0]))
    a = RC.rgd_standard_metric_p1(prob, [u0, v0], 12)
    b = RC.als_cca(Sxx, Syy, Sxy, u0, v0, 12)
    for (u1, v1), (u2, v2) in zip(a, b):
        assert np.max(np.abs(u1 - u2)) < 1e-10 and np.max(np.abs(v1 - v2)) < 1e-10
    # and the iteration does reach the top correlation (rate (sigma_2/sigma_1)^2)
    sig, U, V = cca_qr(P["X64"], P["Y64"], 0.1, 0.1, 1)
    u, v = RC.als_cca(Sxx, Syy, Sxy, u0, v0, 1500)[-1]
    assert abs(abs((u.T @ Sxy @ v).item()) - sig[0]) < 1e-9


def test_rgd_p1_is_power_method_fda():
    P = lda_problem(300, 6, 3, dtype="f64", seed=9)
    SB, Sw = scatters(P["X64"], P["y"], 3)
    Swl = Sw + 0.1 * np.eye(6)
    w0 = np.random.default_rng(1).standard_normal((6, 1))
    prob = FDAProblem(SB, Swl, np.array([1.0]))
    a = RC.rgd_standard_metric_p1(prob, [w0], 10)
    b = RC.power_fda(SB, Swl, w0, 10)
    for (w1,), w2 in zip(a, b):
        assert np.max(np.abs(w1 - w2)) < 1e-10


def test_preconditioning_orders_iteration_counts():
    """M = Sigma needs fewer iterations than the sketch, which needs far fewer
    than M = I on ill-conditioned views (Sec. 6.1-6.2 observations)."""
    rng = np.random.default_rng(1)
    n, dx, dy = 3000, 20, 16
    Z = rng.standard_normal((n, 3)) * np.array([1.0, 0.45, 0.2])
    c = lambda d: 10.0 ** (-3 * np.arange(d) / (d - 1))
    X = (Z @ rng.standard_normal((3, dx)) + 0.3 * rng.standard_normal((n, dx))) * c(dx)
    Y = (Z @ rng.standard_normal((3, dy)) + 0.3 * rng.standard_normal((n, dy))) * c(dy)
    lam, k, s = 1e-6, 2, 400
    h, g = R.countsketch_hash(n, s, seed=1)
    SX, SY = countsketch_apply(X, h, g, s), countsketch_apply(Y, h, g, s)
    mu = default_mu(k)
    it = {m: RC.cca_algorithm1(X, Y, lam, lam, k, mu, SX, SY, gtol=1e-8, max_iter=1000, metric=m)["iters"]
          for m in ("exact", "sketch", "identity")}
    assert it["exact"] <= it["sketch"]
    assert it["sketch"] * 3 < it["identity"]


def test_algorithm2_small():
    P = lda_problem(2000, 15, 5, dtype="f64", seed=2)
    X, y = P["X64"], P["y"]
    lam, k, s = 1e-3, 4, 45
    h, g = R.countsketch_hash(2000, s, seed=5)
    mu = default_mu(k)
    res = RC.fda_algorithm2(X, y, 5, lam, k, mu, RC.sketch_countsketch(h, g, s), gtol=1e-10)
    rho, _ = lda_geneig(X, y, 5, lam, k)
    assert res["status"] in ("converged", "stalled")
    assert np.max(np.abs(res["rho"] - rho) / rho) < 1e-9


def test_polar_retraction_variant():
    """The polar-retraction RCG (Table 1 polar retraction; start normalized by
    x (x^T B x)^{-1/2}) reaches the same closed form.  Its start is the B-polar
    factor of x: on the manifold, with x_new^T B x symmetric positive
    definite; and it agrees with the QR retraction to first order in t."""
    from oracle import geometry as G
    P = cca_latent_problem(1500, 12, 9, latent=4, seed=3, latent_scale=[1.0, 0.6, 0.35, 0.2])
    lam, k = 1e-2, 3
    Sxx, Syy, Sxy = sigmas(P["X64"], P["Y64"], lam, lam)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((12, k))
    xn = RC._normalize(x, Sxx, "polar")
    assert np.max(np.abs(xn.T @ Sxx @ xn - np.eye(k))) < 1e-12
    S = xn.T @ Sxx @ x
    assert np.max(np.abs(S - S.T)) < 1e-12 and np.min(np.linalg.eigvalsh(S)) > 0
    xi = G.proj_tangent(xn, Sxx, np.eye(12), rng.standard_normal((12, k)))
    for t in (1e-3, 1e-4):
        d = np.max(np.abs(G.retr_polar(xn, Sxx, t * xi) - G.retr_qr(xn, Sxx, t * xi)))
        assert d < 50 * t * t * np.max(np.abs(xi)) ** 2 + 1e-13
    prob = CCAProblem(Sxx, Syy, Sxy, default_mu(k))
    y0 = rng.standard_normal((9, k))
    res = RC.rcg(prob, [Sxx, Syy], [x, y0], max_iter=3000, gtol=1e-10, retraction="polar")
    U, V = res["points"]
    sig, _, _ = cca_qr(P["X64"], P["Y64"], lam, lam, k)
    assert res["status"] in ("converged", "stalled")
    assert np.max(np.abs(np.diag(U.T @ Sxy @ V) - sig) / sig) < 1e-9
