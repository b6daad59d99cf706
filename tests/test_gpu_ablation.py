"""Preconditioner ablations of Sec. 6 on the GPU: the metric M = I (no
preconditioning) and M = Sigma = Z^T Z + lambda I (the exact covariance)
against the sketched M = R^T R.

The metric changes the path of the iteration, not its solution (Thm 4.1: the
critical points are the same), so every variant must reach the oracle's
correlations.  The conditioning of the Riemannian Hessian at the optimum is
best with M = Sigma and worst with M = I (Thm 4.4, Cor. 4.5), which on
ill-conditioned data shows in the iteration counts: M = Sigma <= sketch <=
M = I.

The polar retraction (Table 1) replaces the Cholesky factor of the
retraction by the inverse square root of the k x k Gram; the GPU iterates
must follow the oracle's RCG run with the same retraction.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel
from oracle import cca as OC
from oracle import rcg as ORCG
from oracle.precond import precond_R
from oracle.problems import CCAProblem
from oracle.sketch import countsketch_apply
from synth import cca_latent_problem, countsketch_draws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


def _solve(gb, P, n, dx, dy, k, lam, sketch, s):
    o = gb.default_options(sketch=sketch, s=s, max_iter=30000, gtol=0.0, rtol=1e-12, check_every=8)
    plan = gb.cca_plan(n, dx, dy, k, "f64", o)
    gb.cca_precondition(plan, to_dev(P["X"], "f64"), to_dev(P["Y"], "f64"), lam, lam)
    sig, U, V, info = gb.cca_solve(plan)
    plan.close()
    return np64(sig), info


def test_metric_ablation_reaches_the_same_solution(gb):
    """n = 3000, dx = 60, dy = 40, k = 4, columns scaled from 1 to 1e-2
    (kappa(X^T X) ~ 1e4): all three metrics reach the correlations within
    1e-8, and the iteration counts follow the Hessian conditioning."""
    n, dx, dy, k, lam = 3000, 60, 40, 4, 1e-3
    P = cca_latent_problem(n, dx, dy, latent=8, dtype="f64", seed=5, colscale=(1.0, 1e-2),
                           latent_scale=[1.0, 0.8, 0.6, 0.45, 0.3, 0.2, 0.15, 0.1])
    ref, _, _ = OC.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    iters = {}
    for name, sk in (("exact", gb.EXACT), ("sketch", gb.COUNTSKETCH), ("identity", gb.IDENTITY)):
        sig, info = _solve(gb, P, n, dx, dy, k, lam, sk, 400)
        assert info["status"] == gb.OK, (name, info)
        assert rel(sig, ref) < 1e-8, (name, sig, ref, info)
        iters[name] = info["iters"]
    assert iters["exact"] <= iters["sketch"] <= iters["identity"], iters


def test_exact_metric_needs_fp64_cca(gb):
    """M = Sigma forms Z^T Z in FP64 from the stored data: plans of other
    precisions or of FDA report UNSUPPORTED instead of running."""
    n, dx, dy, k = 500, 20, 10, 2
    for dt in ("f32", "bf16"):
        with pytest.raises(gb.GbccaError) as e:
            gb.cca_plan(n, dx, dy, k, dt, gb.default_options(sketch=gb.EXACT, s=100))
        assert e.value.code == gb.ERR_UNSUPPORTED, str(e.value)
    with pytest.raises(gb.GbccaError) as e:
        gb.lda_plan(n, dx, 3, 2, "f64", gb.default_options(sketch=gb.EXACT, s=100))
    assert e.value.code == gb.ERR_UNSUPPORTED, str(e.value)


def test_polar_retraction_trajectory(gb):
    """Same start, same sketch metric, polar retraction: the GPU iterates
    follow the oracle's Riemannian CG with the polar retraction (same
    line-search decisions) for 25 iterations, and the solve converges."""
    import torch
    n, dx, dy, k, lam, s = 1500, 20, 16, 3, 1e-2, 144
    P = cca_latent_problem(n, dx, dy, latent=4, noise=0.6, dtype="f64", seed=8,
                           latent_scale=[1.0, 0.6, 0.35, 0.2])
    h, g = countsketch_draws(n, s, seed=9)
    iters = 25
    o = gb.default_options(s=s, warm_start=0, max_iter=iters, gtol=0.0, retraction=1)
    plan = gb.cca_plan(n, dx, dy, k, "f64", o)
    gb.cca_precondition(plan, to_dev(P["X"], "f64"), to_dev(P["Y"], "f64"), lam, lam,
                        torch.from_numpy(h).cuda(), torch.from_numpy(g).cuda())
    rng = np.random.default_rng(1)
    U0, V0 = rng.standard_normal((dx, k)), rng.standard_normal((dy, k))
    gb.cca_solve(plan, mu=list(OC.default_mu(k)), U=torch.from_numpy(U0.copy()).cuda(),
                 V=torch.from_numpy(V0.copy()).cuda())
    hist = np64(gb.query(plan, gb.Q_HISTORY)).reshape(-1, 3)[: iters + 1]
    plan.close()
    SX, SY = countsketch_apply(P["X64"], h, g, s), countsketch_apply(P["Y64"], h, g, s)
    Rx, Ry = precond_R(SX, lam), precond_R(SY, lam)
    Sxx, Syy, Sxy = OC.sigmas(P["X64"], P["Y64"], lam, lam)
    prob = CCAProblem(Sxx, Syy, Sxy, OC.default_mu(k))
    res = ORCG.rcg(prob, [Rx.T @ Rx, Ry.T @ Ry], [U0, V0], max_iter=iters, gtol=0.0, retraction="polar")
    ho = np.array(res["history"])
    m = min(len(ho), iters + 1)
    assert np.max(np.abs(hist[:m, 0] - ho[:m, 0]) / np.abs(ho[:m, 0])) < 1e-10   # f
    assert np.max(np.abs(hist[1:m, 2] - ho[1:m, 2]) / np.abs(ho[1:m, 2])) < 1e-8  # accepted steps
    assert np.max(np.abs(hist[:m, 1] - ho[:m, 1]) / np.abs(ho[:m, 1])) < 1e-6    # ||grad||_M
    # run to convergence with the polar retraction
    o = gb.default_options(s=s, max_iter=5000, gtol=0.0, rtol=1e-10, retraction=1)
    plan = gb.cca_plan(n, dx, dy, k, "f64", o)
    gb.cca_precondition(plan, to_dev(P["X"], "f64"), to_dev(P["Y"], "f64"), lam, lam)
    sig, _, _, info = gb.cca_solve(plan)
    plan.close()
    ref, _, _ = OC.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    assert info["status"] == gb.OK, info
    assert rel(np64(sig), ref) < 1e-8, (np64(sig), ref)
