"""GPU parity of the Fisher LDA path (Alg. 2) against the CPU oracle."""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel, subspace_sin, bound_ratio
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


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_fda_pass(gb, dt):
    """Every entry within its own rounding bound.  P = X Phi - C[y] with
    C = (class means) Phi; |P| <= (|X| + |M[y]|) |Phi| entrywise; G = X^T P
    minus the class-mean correction, bounded against (|X| + |M[y]|)^T |P|;
    the Gram against |P|^T |P|.  FP32: W chain over d (+ the FP32 copies of
    Phi and C), G partial sums over 128 rows and class sums over 64-row
    tiles flushed to FP64; FP64: the same chains in FP64.  These are the
    CUDA-core kernels (tensor_cores = 0); the tensor-core pass of FP32 FDA
    plans has its own bound (test_gpu_fp32_pass)."""
    import torch
    n, d, l, k = 5003, 61, 6, 5
    P = lda_problem(n, d, l, dtype=dt, seed=3)
    plan, _, _, _ = _solve(gb, P, n, d, l, k, dt, 1e-2, max_iter=2, tensor_cores=0)
    rng = np.random.default_rng(0)
    Phi = rng.standard_normal((d, 2 * k))
    Gx, _, Gram = gb.fused_pass(plan, torch.from_numpy(Phi).cuda())
    ox, og = OF.lda_pass(P["X64"], P["y"], l, Phi)
    _, means, _, _, _ = OL.class_stats(P["X64"], P["y"], l)
    aZ = np.abs(P["X64"]) + np.abs(means[P["y"]])
    aP = aZ @ np.abs(Phi)
    if dt == "f64":
        gG = gW = 4 * (d + n + 4) * 2.0 ** -53
    else:
        gG, gW = (d + 3 + 128 + 64 + 2) * 2.0 ** -24, (2 * (d + 3) + 64 + 2) * 2.0 ** -24
    assert bound_ratio(np64(Gx), ox, aZ.T @ aP, gG) <= 1.0
    assert bound_ratio(np64(Gram), og, aP.T @ aP, gW) <= 1.0
