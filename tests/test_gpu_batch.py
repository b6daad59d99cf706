"""GPU parity of batched solves (several prepared plans in lockstep, the
tensor-core passes of all of them in one persistent launch) through the C ABI.

The batched pass is the kernel of the single-plan pass with a segment
schedule: each 2-CTA cluster walks contiguous tile ranges of one or more
instances, reloading the Phi image and draining its G accumulators at every
instance boundary.  Its rounding is the single-plan kernel's, except that an
instance's tiles may sit on fewer clusters, so the bound below takes the
worst case of every tile of the instance in one cluster (T = its tiles).

Each instance's batched solve must give the correlations of its own solo
solve within 1e-6 relative (and of the oracle within 1e-6).
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel, bound_ratio, cca_pass_refs
from oracle import cca as OC
from oracle import fused as OF
from oracle import lda as OL
from synth import cca_latent_problem, lda_problem, f32_to_bf16_bits, bf16_bits_to_f32

pytestmark = pytest.mark.gpu

SCALE = [1.0, 0.8, 0.6, 0.45, 0.33, 0.25, 0.18, 0.13, 0.1, 0.07, 0.05, 0.035, 0.025, 0.018, 0.012, 0.008]


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


def bf16_round(x):
    return bf16_bits_to_f32(f32_to_bf16_bits(np.asarray(x, dtype=np.float32))).astype(np.float64)


def split_round(P):
    hi = bf16_round(P)
    return hi + bf16_round(P - hi)


def gamma_batched(rows, d, fp32):
    """Single-plan bound with every 64-row tile of the instance in one
    cluster; FP32 data adds the representation of Z twice and the hi/lo row
    sum (see test_gpu_fp32_pass)."""
    T = -(-rows // 64)
    g = 2.0 ** -17 + 2.0 ** -23 * (2 * (d / 16 + 2) + 2 * (4 * T + 1) + 4 + 2)  # + the halves' partial-W sum
    if fp32:
        g += 2 * 2.0 ** -17 + 2 * 2.0 ** -23
    return g


# (n, dx, dy, k, storage): ragged sizes, both Phi image widths (2k <= 20 and
# 2k = 24), one-pair and four-pair views, FP32 data through the interleaved
# copy, k = 20 (two column groups, two table entries for one plan), and
# views wider than 512 (the second batched launch, in 4-CTA clusters)
SHAPES = [(9001, 200, 120, 5, "bf16"), (4097, 64, 40, 10, "bf16"), (20000, 512, 296, 12, "bf16"),
          (3001, 96, 80, 4, "f32"), (150, 24, 16, 3, "bf16"), (6007, 160, 128, 20, "bf16"),
          (5003, 768, 200, 6, "bf16"), (2001, 1024, 64, 3, "f32")]


def _make(gb, shapes, seed0=0, **opt):
    plans, probs = [], []
    for i, (n, dx, dy, k, dt) in enumerate(shapes):
        P = cca_latent_problem(n, dx, dy, latent=16, dtype=dt, seed=seed0 + i, latent_scale=SCALE,
                               colscale=(1.0, 1e-2))
        o = gb.default_options(**opt)
        plan = gb.cca_plan(n, dx, dy, k, dt, o)
        gb.cca_precondition(plan, to_dev(P["X"], dt), to_dev(P["Y"], dt), 1e-3, 1e-3)
        plans.append(plan)
        probs.append(P)
    return plans, probs


@pytest.mark.parametrize("clusters", [0, 3, 76])
def test_batched_pass_matches_oracle(gb, clusters):
    """One batched pass over five instances: every entry of every G and Gram
    within its own bound, for the tuned schedule and for 3 and 76 clusters
    (instances split over many clusters, and many instances per cluster)."""
    import torch
    plans, probs = _make(gb, SHAPES)
    batch = gb.Batch(plans, gb.default_batch_options(clusters=clusters))
    rng = np.random.default_rng(7)
    Px, Py = [], []
    for (n, dx, dy, k, dt) in SHAPES:
        Px.append(rng.standard_normal((dx, 2 * k)) / np.sqrt(dx))
        Py.append(rng.standard_normal((dy, 2 * k)) / np.sqrt(dy))
    G, Gram = gb.batch_fused_pass(batch, [torch.from_numpy(a).cuda() for a in Px],
                                  [torch.from_numpy(a).cuda() for a in Py])
    torch.cuda.synchronize()
    for i, (n, dx, dy, k, dt) in enumerate(SHAPES):
        P = probs[i]
        pxr, pyr = split_round(Px[i]), split_round(Py[i])
        ox, oy, og = OF.cca_pass(P["X64"], P["Y64"], pxr, pyr)
        rx, ry, rg, _ = cca_pass_refs(P["X64"], P["Y64"], pxr, pyr)
        g = np64(G[i])
        gam = gamma_batched(2 * n if dt == "f32" else n, max(dx, dy), dt == "f32")
        for name, got, exp, ref in (("Gx", g[:dx], ox, rx), ("Gy", g[dx:], oy, ry), ("Gram", np64(Gram[i]), og, rg)):
            r = bound_ratio(got, exp, ref, gam)
            assert r <= 1.0, (i, name, r)
    batch.close()
    for p in plans:
        p.close()


def test_batch_solve_matches_solo_solves(gb):
    """Seven plans in one batch: six served by the batched launches (BF16
    and FP32 data, 2k = 30 in two column groups, and a 600-wide view in the
    4-CTA launch) and an FDA plan (its own FP32 pass on its branch).  Each
    result equals its solo solve within 1e-6 and the oracle within 1e-6."""
    import torch
    shapes = [(9001, 200, 120, 5, "bf16"), (4097, 64, 40, 10, "bf16"), (20000, 512, 296, 12, "bf16"),
              (3001, 96, 80, 4, "f32"), (5000, 104, 88, 15, "bf16"), (7000, 600, 64, 4, "bf16")]
    opt = dict(max_iter=3000, gtol=0.0, rtol=1e-7, check_every=8, refine=2)
    plans, probs = _make(gb, shapes, seed0=20, **opt)
    solo = []
    for plan in plans:
        sig, _, _, info = gb.cca_solve(plan)
        assert info["status"] == gb.OK, info
        solo.append(np64(sig))
    n, d, l, k = 8000, 60, 6, 5
    PL = lda_problem(n, d, l, dtype="f32", seed=3)
    lplan = gb.lda_plan(n, d, l, k, "f32", gb.default_options(max_iter=3000, gtol=0.0, rtol=1e-7, check_every=8))
    Xl, yl = to_dev(PL["X"], "f32"), torch.from_numpy(PL["y"]).cuda()
    rho, _, info = gb.lda_solve(lplan, Xl, yl, 1e-2)
    assert info["status"] == gb.OK, info
    solo.append(np64(rho))
    allp = plans + [lplan]
    batch = gb.Batch(allp)
    res, report = gb.batch_solve(batch)
    assert report["batched_plans"] == 6, report
    assert report["batched_pass_ms"] > 0 and report["clusters"] >= 1, report
    for i, (val, _, _, info) in enumerate(res):
        assert info["status"] == gb.OK, (i, info)
        assert rel(np64(val), solo[i]) < 1e-6, (i, np64(val), solo[i])
    for i, (nn, dx, dy, kk, dt) in enumerate(shapes):
        ref, _, _ = OC.cca_qr(probs[i]["X64"], probs[i]["Y64"], 1e-3, 1e-3, kk)
        assert rel(np64(res[i][0]), ref) < 1e-6, (i, np64(res[i][0]), ref)
    ref, _ = OL.lda_geneig(PL["X64"], PL["y"], l, 1e-2, k)
    assert rel(np64(res[-1][0]), ref) < 1e-6
    # later solves of the same batch (tuned schedule, graphs captured again as
    # plans finish) repeat each other exactly; the first one differs only by
    # the schedule trials, which round the start point's Phi image once more
    res2, _ = gb.batch_solve(batch)
    res3, _ = gb.batch_solve(batch)
    for i in range(len(allp)):
        assert rel(np64(res2[i][0]), np64(res[i][0])) < 1e-6, i
        assert np.array_equal(np64(res3[i][0]), np64(res2[i][0])), i
    batch.close()
    for p in allp:
        p.close()


def test_batch_rejects_unprepared_plans(gb):
    """A plan not bound to its data cannot join a batch (GBCCA_ERR_STATE), and
    the same plan twice is refused."""
    plan = gb.cca_plan(1000, 20, 10, 2, "bf16", gb.default_options())
    with pytest.raises(gb.GbccaError) as e:
        gb.Batch([plan])
    assert e.value.code == gb.ERR_STATE
    plans, _ = _make(gb, [(500, 20, 10, 2, "bf16")])
    with pytest.raises(gb.GbccaError) as e:
        gb.Batch([plans[0], plans[0]])
    assert e.value.code == gb.ERR_INVALID_ARG
    plan.close()
    plans[0].close()
