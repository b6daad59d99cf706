"""GPU parity of the Fisher LDA path (Alg. 2) against the CPU oracle."""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel, subspace_sin
from oracle import lda as OL
from oracle import fused as OF
from oracle.sketch import countsketch_apply
from synth import lda_problem, countsketch_draws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


def _solve(gb, P, n, d, l, k, dt, lam, **opt):
    import torch
    o = gb.default_options(**opt)
    plan = gb.lda_plan(n, d, l, k, dt, o)
    X = to_dev(P["X"], dt)
    y = torch.from_numpy(P["y"]).cuda()
    rho, W, info = gb.lda_solve(plan, X, y, lam)
    return plan, np64(rho), np64(W), info


def test_class_means_and_sketch_fp64(gb):
    import torch
    n, d, l, k, s = 3001, 37, 5, 4, 120
    P = lda_problem(n, d, l, dtype="f64", seed=1)
    h, g = countsketch_draws(n, s, seed=2)
    plan = gb.lda_plan(n, d, l, k, "f64", gb.default_options(s=s, max_iter=5))
    X = to_dev(P["X"], "f64")
    y = torch.from_numpy(P["y"]).cuda()
    gb.lda_solve(plan, X, y, 1e-2, sketch_h=torch.from_numpy(h).cuda(), sketch_g=torch.from_numpy(g).cuda())
    counts, means, m, Yhat, Xhat = OL.class_stats(P["X64"], P["y"], l)
    assert rel(np64(gb.query(plan, gb.Q_CLASS_MEANS)).reshape(l, d), means) < 1e-13
    SX = np64(gb.query(plan, gb.Q_SKETCH_X)).reshape(s, d)
    assert rel(SX, countsketch_apply(Xhat, h, g, s)) < 1e-12


@pytest.mark.parametrize("dt,tol", [("f64", 1e-12), ("f32", 5e-5)])
def test_fda_pass(gb, dt, tol):
    import torch
    n, d, l, k = 5003, 61, 6, 5
    P = lda_problem(n, d, l, dtype=dt, seed=3)
    plan, _, _, _ = _solve(gb, P, n, d, l, k, dt, 1e-2, max_iter=2)
    rng = np.random.default_rng(0)
    Phi = rng.standard_normal((d, 2 * k))
    Gx, _, Gram = gb.fused_pass(plan, torch.from_numpy(Phi).cuda())
    ox, og = OF.lda_pass(P["X64"], P["y"], l, Phi)
    assert rel(np64(Gx), ox) < tol
    assert rel(np64(Gram), og) < tol


def test_lda_solve_fp64(gb):
    n, d, l, k, lam = 3000, 20, 5, 4, 1e-3
    P = lda_problem(n, d, l, dtype="f64", seed=4)
    _, rho, W, info = _solve(gb, P, n, d, l, k, "f64", lam, max_iter=3000, gtol=1e-11, s=60)
    ref, Wo = OL.lda_geneig(P["X64"], P["y"], l, lam, k)
    assert rel(rho, ref) < 1e-8, (rho, ref, info)
    SB, Sw = OL.scatters(P["X64"], P["y"], l)
    Swl = Sw + lam * np.eye(d)
    assert np.max(np.abs(W.T @ Swl @ W - np.eye(k))) < 1e-8
    # eigenvalue errors are quadratic in the subspace angle: 1e-8 on rho allows
    # angles of order 1e-5 for the closest eigenvalue gaps of this problem
    assert subspace_sin(W, Wo, Swl) < 1e-5


def test_lda_solve_f32_refined(gb):
    n, d, l, k, lam = 20000, 96, 8, 7, 1e-3
    P = lda_problem(n, d, l, dtype="f32", seed=5)
    _, rho, W, info = _solve(gb, P, n, d, l, k, "f32", lam, max_iter=1000, gtol=1e-6)
    ref, _ = OL.lda_geneig(P["X64"], P["y"], l, lam, k)
    assert rel(rho, ref) < 1e-6, (rho, ref, info)
