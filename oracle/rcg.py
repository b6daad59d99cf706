"""Reference Riemannian CG, Algorithms 1 and 2, and the p = 1 special cases.

TEST INFRASTRUCTURE ONLY (see package docstring).

Riemannian CG (Sec. 2.2 components; Alg. 1 step 8, Alg. 2 step 9).  The paper
defers step rule, CG coefficient and stopping to manopt defaults (Sec. 6.1);
this module fixes one reading of them, the same one the library implements:

  * direction: eta_0 = -grad; then eta = -grad + beta T(eta_prev) with the
    Hestenes-Stiefel coefficient clipped at zero,
        beta = max(0, g(grad, y) / g(T(eta_prev), y)),  y = grad - T(grad_prev),
    T = projection onto the new tangent space (Table 1 vector transport);
    if g(grad, eta) >= 0 the direction restarts as -grad.
  * line search along t -> R_X(t eta) (QR retraction, or the polar one on
    request): first trial
    t = 1 / ||eta||_M on the first iteration, else t_prev * df_prev / df
    (df = g(grad, eta)); Armijo backtracking with c1 = 1e-4 halving t, at most
    25 trials (Sec. 6.1: manopt rejects a step after 25); if the first trial
    already passes, t doubles while the cost keeps decreasing and Armijo holds
    (at most 10 doublings).  A step with no accepted trial ends the run with
    status "stalled": no trial could lower f, i.e. f has reached its rounding
    floor.
  * stop when ||grad||_M <= gtol * ||grad_0||_M or after max_iter iterations.

Also here: RGD with the standard metric and step 1 / (u^T Sxy v) for p = 1,
which Sec. 6.2 states is ALS for CCA (Golub-Zha) and the power method for FDA;
and end-to-end Algorithms 1 and 2 (sketch, warm start, qf_B, RCG with M).

Parity: pinned by convergence to the closed forms (oracle.cca, oracle.lda), by
the RGD == ALS / power-method identity, and by the M = Sigma / sketch / M = I
ordering of iteration counts (tests/test_oracle_rcg.py).
"""
from __future__ import annotations

import numpy as np

from . import geometry as G
from .cca import sigmas, cca_whiten
from .lda import class_stats
from .precond import precond_R
from .problems import CCAProblem, FDAProblem
from .sketch import countsketch_apply, srht_apply

C1 = 1e-4
MAX_LS = 25
MAX_EXPAND = 10


def _retr(pts, Bs, etas, t, retraction="qr"):
    f = G.retr_polar if retraction == "polar" else G.retr_qr
    return [f(x, B, t * e) for x, B, e in zip(pts, Bs, etas)]


def _normalize(x, B, retraction):
    """Starting point on St_B: qf_B (the QR retraction at a zero step), or for
    the polar retraction its own zero-step map x (x^T B x)^{-1/2}."""
    if retraction == "polar":
        w, Q = np.linalg.eigh(x.T @ B @ x)
        return x @ ((Q / np.sqrt(w)) @ Q.T)
    return G.retr_chol(x, B, np.zeros_like(x))


def rcg(problem, Ms, X0s, max_iter=1000, gtol=1e-8, record=False, retraction="qr"):
    """Riemannian CG on the product of St_{B_i} with metrics M_i.

    retraction: "qr" (Table 1 QR retraction) or "polar" (Table 1 polar
    retraction); the starting point is normalized by the same map.
    Returns dict(points, iters, history=[(f, ||grad||_M, t), ...], status).
    """
    Bs = problem.Bs
    pts = [_normalize(x, B, retraction) for x, B in zip(X0s, Bs)]
    f = problem.cost(pts)
    eg = problem.egrad(pts)
    grads = [G.rgrad(x, B, M, g) for x, B, M, g in zip(pts, Bs, Ms, eg)]
    gn = np.sqrt(sum(G.metric(M, g, g) for M, g in zip(Ms, grads)))
    gn0 = gn
    etas = [-g for g in grads]
    t_prev = df_prev = None
    hist = [(f, gn, 0.0)]
    status = "maxiter"
    it = 0
    for it in range(max_iter):
        if gn <= gtol * gn0:
            status = "converged"
            break
        df = sum(float(np.sum(g * e)) for g, e in zip(eg, etas))
        if df >= 0:
            etas = [-g for g in grads]
            df = -gn * gn
        if t_prev is None:
            t = 1.0 / np.sqrt(sum(G.metric(M, e, e) for M, e in zip(Ms, etas)))
        else:
            t = t_prev * df_prev / df
        ok = False
        for j in range(MAX_LS):
            ft = problem.cost(_retr(pts, Bs, etas, t, retraction))
            if ft <= f + C1 * t * df:
                ok = True
                break
            t *= 0.5
        if not ok:
            status = "stalled"  # no trial decreased f: the rounding floor of f
            break
        if j == 0:
            for _ in range(MAX_EXPAND):
                t2 = 2.0 * t
                f2 = problem.cost(_retr(pts, Bs, etas, t2, retraction))
                if f2 < ft and f2 <= f + C1 * t2 * df:
                    t, ft = t2, f2
                else:
                    break
        new = _retr(pts, Bs, etas, t, retraction)
        eg = problem.egrad(new)
        g_new = [G.rgrad(x, B, M, g) for x, B, M, g in zip(new, Bs, Ms, eg)]
        eta_T = [G.proj_tangent(x, B, M, e) for x, B, M, e in zip(new, Bs, Ms, etas)]
        grad_T = [G.proj_tangent(x, B, M, g) for x, B, M, g in zip(new, Bs, Ms, grads)]
        y = [a - b for a, b in zip(g_new, grad_T)]
        num = sum(G.metric(M, a, b) for M, a, b in zip(Ms, g_new, y))
        den = sum(G.metric(M, a, b) for M, a, b in zip(Ms, eta_T, y))
        beta = max(0.0, num / den) if den != 0.0 else 0.0
        etas = [-a + beta * b for a, b in zip(g_new, eta_T)]
        pts, grads, f = new, g_new, ft
        gn = np.sqrt(sum(G.metric(M, g, g) for M, g in zip(Ms, grads)))
        t_prev, df_prev = t, df
        hist.append((f, gn, t))
    else:
        it = max_iter
    if status == "maxiter" and gn <= gtol * gn0:
        status = "converged"
    return dict(points=pts, iters=it, history=hist, status=status)


def rgd_standard_metric_p1(problem, x0s, iters, mu=1.0):
    """RGD, p = 1, metric M = B, step 1 / (mu * x^T A x') (Sec. 6.2's ALS link)."""
    Bs = problem.Bs
    pts = [G.retr_chol(x, B, np.zeros_like(x)) for x, B in zip(x0s, Bs)]
    out = [pts]
    for _ in range(iters):
        eg = problem.egrad(pts)
        grads = [G.rgrad(x, B, B, g) for x, B, g in zip(pts, Bs, eg)]
        alpha = 1.0 / (-problem.cost(pts) * (2.0 if isinstance(problem, FDAProblem) else 1.0))
        pts = [G.retr_qr(x, B, -alpha * g) for x, B, g in zip(pts, Bs, grads)]
        out.append(pts)
    return out


def als_cca(Sxx, Syy, Sxy, u0, v0, iters):
    """Simultaneous ALS / power iteration for the top canonical pair:
    u <- Sxx^{-1} Sxy v, v <- Syy^{-1} Sxy^T u, each normalized in its B-norm."""
    def nrm(z, B):
        return z / np.sqrt((z.T @ B @ z).item())
    u, v = nrm(u0, Sxx), nrm(v0, Syy)
    out = [(u, v)]
    for _ in range(iters):
        u, v = nrm(np.linalg.solve(Sxx, Sxy @ v), Sxx), nrm(np.linalg.solve(Syy, Sxy.T @ u), Syy)
        out.append((u, v))
    return out


def power_fda(SB, Swl, w0, iters):
    """Power method on (S_w + lambda I)^{-1} S_B, B-normalized."""
    def nrm(z):
        return z / np.sqrt((z.T @ Swl @ z).item())
    w = nrm(w0)
    out = [w]
    for _ in range(iters):
        w = nrm(np.linalg.solve(Swl, SB @ w))
        out.append(w)
    return out


def cca_algorithm1(X, Y, lx, ly, k, mu, SX, SY, max_iter=1000, gtol=1e-8, metric="sketch"):
    """Alg. 1 given the sketched views SX = S X, SY = S Y (same S for both).

    metric: "sketch" (M = (SX)^T SX + lambda I), "exact" (M = Sigma), "identity".
    """
    Sxx, Syy, Sxy = sigmas(X, Y, lx, ly)
    _, U0, V0 = cca_whiten(SX, SY, lx, ly, k)  # exact-cca on the sketch
    if metric == "sketch":
        Rx, Ry = precond_R(SX, lx), precond_R(SY, ly)
        Ms = [Rx.T @ Rx, Ry.T @ Ry]
    elif metric == "exact":
        Ms = [Sxx, Syy]
    else:
        Ms = [np.eye(Sxx.shape[0]), np.eye(Syy.shape[0])]
    prob = CCAProblem(Sxx, Syy, Sxy, mu)
    res = rcg(prob, Ms, [U0, V0], max_iter=max_iter, gtol=gtol)
    U, V = res["points"]
    res["sigma"] = np.diag(U.T @ Sxy @ V).copy()
    res["f"] = prob.cost(res["points"])
    return res


def fda_algorithm2(X, y, l, lam, k, mu, sketch_fn, max_iter=1000, gtol=1e-8, metric="sketch"):
    """Alg. 2: sketch Xhat with ``sketch_fn`` (S Xhat), warm start from the
    exact FDA of the sketch, RCG with M = (S Xhat)^T (S Xhat) + lambda I."""
    _, _, _, Yhat, Xhat = class_stats(X, y, l)
    SB = Yhat.T @ Yhat
    d = Xhat.shape[1]
    Swl = Xhat.T @ Xhat + lam * np.eye(d)
    XS = sketch_fn(Xhat)
    R = precond_R(XS, lam)
    Msk = R.T @ R
    # exact-fda on the sketch: leading generalized eigenvectors of (S_B, Msk)
    import scipy.linalg as sl
    w, Vv = sl.eigh(SB, Msk)
    W0 = Vv[:, np.argsort(w)[::-1][:k]]
    Ms = [Msk if metric == "sketch" else (Swl if metric == "exact" else np.eye(d))]
    prob = FDAProblem(SB, Swl, mu)
    res = rcg(prob, Ms, [W0], max_iter=max_iter, gtol=gtol)
    (W,) = res["points"]
    res["rho"] = np.diag(W.T @ SB @ W).copy()
    res["f"] = prob.cost(res["points"])
    return res


def sketch_countsketch(h, g, s):
    return lambda Z: countsketch_apply(Z, h, g, s)


def sketch_srht(D, rows):
    return lambda Z: srht_apply(Z, D, rows)
