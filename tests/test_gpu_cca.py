"""GPU parity of the CCA hot path (Alg. 1) against the CPU oracle, through the C ABI.

Tolerances: FP64 data -> results within 1e-8 relative of the oracle (sketch,
R, pass: ~1e-12, set by FP64 rounding of sums of length <= n); BF16/FP32
data -> pass outputs within the FP32-accumulation bound below, canonical
correlations within 1e-6 relative after the FP64 Rayleigh-Ritz refinement.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel, subspace_sin, bound_ratio, cca_pass_refs
from oracle import cca as OC
from oracle import fused as OF
from oracle import rcg as ORCG
from oracle import rng as ORNG
from oracle.precond import precond_R
from oracle.sketch import countsketch_apply, srht_apply
from synth import cca_latent_problem, countsketch_draws, srht_draws

pytestmark = pytest.mark.gpu

SEP = [1.0, 0.6, 0.35, 0.2]


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


def _plan(gb, P, n, dx, dy, k, dt, lam, sketch=0, s=0, h=None, g=None, **opt):
    o = gb.default_options(sketch=sketch, s=s, **opt)
    plan = gb.cca_plan(n, dx, dy, k, dt, o)
    X, Y = to_dev(P["X"], dt), to_dev(P["Y"], dt)
    gb.cca_precondition(plan, X, Y, lam, lam, h, g)
    return plan, X, Y


def test_countsketch_explicit_draws_fp64(gb):
    import torch
    n, dx, dy, s = 3001, 37, 29, 200  # ragged sizes: not multiples of any tile
    P = cca_latent_problem(n, dx, dy, latent=5, dtype="f64", seed=1)
    h, g = countsketch_draws(n, s, seed=4)
    plan, _, _ = _plan(gb, P, n, dx, dy, 3, "f64", 1e-2, s=s, h=torch.from_numpy(h).cuda(),
                       g=torch.from_numpy(g).cuda())
    SX = np64(gb.query(plan, gb.Q_SKETCH_X)).reshape(s, dx)
    SY = np64(gb.query(plan, gb.Q_SKETCH_Y)).reshape(s, dy)
    assert rel(SX, countsketch_apply(P["X64"], h, g, s)) < 1e-13
    assert rel(SY, countsketch_apply(P["Y64"], h, g, s)) < 1e-13
    # R factor: R^T R = (SX)^T SX + lambda I and equal to the oracle's QR factor
    Rx = np64(gb.query(plan, gb.Q_R_X)).reshape(dx, dx)
    Ro = precond_R(countsketch_apply(P["X64"], h, g, s), 1e-2)
    assert rel(Rx, Ro) < 1e-10
    assert np.allclose(np.tril(Rx, -1), 0)


def test_countsketch_library_draws_bitexact(gb):
    n, s, seed = 100003, 977, 12345
    h, g = gb.sketch_draws(gb.COUNTSKETCH, n, s, seed)
    ho, go = ORNG.countsketch_hash(n, s, seed)
    assert np.array_equal(h.cpu().numpy(), ho)
    assert np.array_equal(g.cpu().numpy(), go)


def test_srht_library_draws_bitexact(gb):
    for m, s in ((12, 300), (13, 1000)):
        rows, signs = gb.sketch_draws(gb.SRHT, 1 << m, s, 77)
        assert np.array_equal(rows.cpu().numpy(), ORNG.srht_rows(1 << m, s, 77))
        assert np.array_equal(signs.cpu().numpy(), ORNG.srht_signs(1 << m, 77))


@pytest.mark.parametrize("dt,tol", [("f64", 1e-12), ("f32", 2e-6), ("bf16", 2e-6)])
def test_srht_sketch(gb, dt, tol):
    import torch
    n, dx, dy, s = 5000, 40, 33, 300   # n_pad = 8192 = 2^13 -> two stages
    P = cca_latent_problem(n, dx, dy, latent=4, dtype=dt, seed=2)
    D, rows = srht_draws(8192, s, seed=3)
    plan, _, _ = _plan(gb, P, n, dx, dy, 2, dt, 1e-2, sketch=gb.SRHT, s=s,
                       h=torch.from_numpy(rows).cuda(), g=torch.from_numpy(D).cuda())
    SX = np64(gb.query(plan, gb.Q_SKETCH_X)).reshape(s, dx)
    assert rel(SX, srht_apply(P["X64"], D, rows)) < tol


def gamma_cores(dt, n, d):
    """Entrywise bounds of the CUDA-core pass, against the sums of |terms|.
    FP32 accumulation (BF16/FP32 data): Phi rounded to FP32 (1 rounding), W
    by an FMA chain over d columns (d roundings), G by FP32 partial sums over
    128 rows flushed to FP64 (128 + 2), the Gram by FP32 sums over 64-row
    tiles of W products (64 + 2, and W's own error twice).  FP64 data: the
    same chains in FP64 over at most d + n terms."""
    if dt == "f64":
        g = 4 * (d + n + 4) * 2.0 ** -53
        return g, g
    return (d + 1 + 128 + 2) * 2.0 ** -24, (2 * (d + 1) + 64 + 2) * 2.0 ** -24


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_fused_pass(gb, dt):
    """Every entry of Gx, Gy and the Gram within its own rounding bound."""
    import torch
    n, dx, dy, k = 4099, 70, 45, 5
    P = cca_latent_problem(n, dx, dy, latent=6, dtype=dt, seed=5, colscale=(1.0, 1e-3))
    plan, _, _ = _plan(gb, P, n, dx, dy, k, dt, 1e-2)
    rng = np.random.default_rng(0)
    Px, Py = rng.standard_normal((dx, 2 * k)), rng.standard_normal((dy, 2 * k))
    Gx, Gy, Gram = gb.fused_pass(plan, torch.from_numpy(Px).cuda(), torch.from_numpy(Py).cuda())
    ox, oy, og = OF.cca_pass(P["X64"], P["Y64"], Px, Py)
    rx, ry, _, aW = cca_pass_refs(P["X64"], P["Y64"], Px, Py)
    gG, gW = gamma_cores(dt, n, max(dx, dy))
    assert bound_ratio(np64(Gx), ox, rx, gG) <= 1.0
    assert bound_ratio(np64(Gy), oy, ry, gG) <= 1.0
    assert bound_ratio(np64(Gram), og, aW.T @ aW, gW) <= 1.0


def test_solve_separated_fp64(gb):
    n, dx, dy, k, lam = 1000, 24, 20, 3, 1e-3
    P = cca_latent_problem(n, dx, dy, latent=4, noise=0.6, dtype="f64", seed=3, latent_scale=SEP)
    plan, _, _ = _plan(gb, P, n, dx, dy, k, "f64", lam, max_iter=2000, gtol=1e-11)
    sig, U, V, info = gb.cca_solve(plan)
    ref, Uo, Vo = OC.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    assert rel(np64(sig), ref) < 1e-9, (np64(sig), ref, info)
    Sxx, Syy, Sxy = OC.sigmas(P["X64"], P["Y64"], lam, lam)
    U, V = np64(U), np64(V)
    assert np.max(np.abs(U.T @ Sxx @ U - np.eye(k))) < 1e-9
    assert np.max(np.abs(U.T @ Sxy @ V - np.diag(ref))) < 1e-9
    assert subspace_sin(U, Uo, Sxx) < 1e-6


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_warm_start_is_sketched_cca(gb, dt):
    """f64: FP64 products; f32: the double-float products of FP32/BF16 plans."""
    import torch
    n, dx, dy, k, lam, s = 2000, 30, 26, 3, 1e-2, 240
    P = cca_latent_problem(n, dx, dy, latent=4, noise=0.6, dtype=dt, seed=6, latent_scale=SEP)
    h, g = countsketch_draws(n, s, seed=7)
    plan, _, _ = _plan(gb, P, n, dx, dy, k, dt, lam, s=s, h=torch.from_numpy(h).cuda(),
                       g=torch.from_numpy(g).cuda())
    SX, SY = countsketch_apply(P["X64"], h, g, s), countsketch_apply(P["Y64"], h, g, s)
    _, Uw, Vw = OC.cca_whiten(SX, SY, lam, lam, k)
    Ug = np64(gb.query(plan, gb.Q_WARM_U)).reshape(dx, k)
    Mx = SX.T @ SX + lam * np.eye(dx)
    assert subspace_sin(Ug, Uw, Mx) < 1e-6


def test_trajectory_matches_reference_rcg(gb):
    """Same start, same sketch metric: the GPU iterates follow the oracle's
    Riemannian CG (same line-search decisions) for the first 25 iterations."""
    import torch
    n, dx, dy, k, lam, s = 1500, 20, 16, 3, 1e-2, 144
    P = cca_latent_problem(n, dx, dy, latent=4, noise=0.6, dtype="f64", seed=8, latent_scale=SEP)
    h, g = countsketch_draws(n, s, seed=9)
    iters = 25
    plan, _, _ = _plan(gb, P, n, dx, dy, k, "f64", lam, s=s, h=torch.from_numpy(h).cuda(),
                       g=torch.from_numpy(g).cuda(), warm_start=0, max_iter=iters, gtol=0.0)
    rng = np.random.default_rng(1)
    U0, V0 = rng.standard_normal((dx, k)), rng.standard_normal((dy, k))
    gb.cca_solve(plan, mu=list(OC.default_mu(k)), U=torch.from_numpy(U0.copy()).cuda(),
                 V=torch.from_numpy(V0.copy()).cuda())
    hist = np64(gb.query(plan, gb.Q_HISTORY)).reshape(-1, 3)[: iters + 1]
    SX, SY = countsketch_apply(P["X64"], h, g, s), countsketch_apply(P["Y64"], h, g, s)
    Rx, Ry = precond_R(SX, lam), precond_R(SY, lam)
    Sxx, Syy, Sxy = OC.sigmas(P["X64"], P["Y64"], lam, lam)
    from oracle.problems import CCAProblem
    prob = CCAProblem(Sxx, Syy, Sxy, OC.default_mu(k))
    res = ORCG.rcg(prob, [Rx.T @ Rx, Ry.T @ Ry], [U0, V0], max_iter=iters, gtol=0.0)
    ho = np.array(res["history"])
    m = min(len(ho), iters + 1)
    assert np.max(np.abs(hist[:m, 0] - ho[:m, 0]) / np.abs(ho[:m, 0])) < 1e-10   # f
    assert np.max(np.abs(hist[1:m, 2] - ho[1:m, 2]) / np.abs(ho[1:m, 2])) < 1e-8  # accepted steps
    assert np.max(np.abs(hist[:m, 1] - ho[:m, 1]) / np.abs(ho[:m, 1])) < 1e-6    # ||grad||_M


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_solve_low_precision_refined(gb, dt):
    n, dx, dy, k, lam = 20000, 64, 48, 4, 1e-4
    P = cca_latent_problem(n, dx, dy, latent=6, noise=0.5, colscale=(1.0, 1e-4), dtype=dt, seed=10,
                           latent_scale=[1.0, 0.7, 0.5, 0.35, 0.25, 0.18])
    plan, _, _ = _plan(gb, P, n, dx, dy, k, dt, lam, sketch=gb.SRHT, max_iter=1000, gtol=1e-7)
    sig, U, V, info = gb.cca_solve(plan)
    ref, _, _ = OC.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    assert rel(np64(sig), ref) < 1e-6, (np64(sig), ref, info)


def test_solve_small_fp64_workload(gb):
    """The plain FP64 workload (n=2000, dx=50, dy=40, k=5, lambda=1e-3, CountSketch
    s=360), run to 1e-10: the Rayleigh-Ritz values of span([U, eta]) change by
    less than 1e-10 at two consecutive checks.  The run must stop on that
    rule, not on the iteration cap, with every correlation within 1e-8."""
    n, dx, dy, k, lam = 2000, 50, 40, 5, 1e-3
    P = cca_latent_problem(n, dx, dy, latent=10, noise=0.5, dtype="f64", seed=0)
    plan, _, _ = _plan(gb, P, n, dx, dy, k, "f64", lam, s=360, max_iter=6000, gtol=0.0, rtol=1e-10, check_every=8)
    sig, U, V, info = gb.cca_solve(plan)
    ref, _, _ = OC.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    assert info["status"] == gb.OK and info["iters"] < 6000, info
    assert rel(np64(sig), ref) < 1e-8, (np64(sig), ref, info)


@pytest.mark.parametrize("dt", ["bf16", "f64"])
def test_graph_replay_matches_direct_launches(gb, dt):
    """Batches of iterations replayed from a captured CUDA graph run the same
    kernels in the same order as direct launches: results, iteration counts and
    the library's launch count agree exactly.  A second precondition with
    copies of X and Y at new addresses must re-capture (the captured TMA
    descriptors and data pointers change) and still give the same results."""
    import torch
    n, dx, dy, k, lam = 20000, 192, 136, 5, 1e-3
    P = cca_latent_problem(n, dx, dy, latent=8, dtype=dt, seed=21)
    out = {}
    for graphs in (0, 1):
        plan, X, Y = _plan(gb, P, n, dx, dy, k, dt, lam, s=1400, max_iter=300, gtol=1e-7, check_every=4,
                           graphs=graphs)
        l0 = gb.launch_count()
        sig, U, V, info = gb.cca_solve(plan)
        torch.cuda.synchronize()
        launches = gb.launch_count() - l0
        out[graphs] = (np64(sig), np64(U), np64(V), info["iters"], launches)
        if graphs:
            X2, Y2 = X.clone(), Y.clone()
            del X, Y
            gb.cca_precondition(plan, X2, Y2, lam, lam)
            sig2, U2, V2, info2 = gb.cca_solve(plan)
            assert np.array_equal(np64(sig2), out[1][0]) and np.array_equal(np64(U2), out[1][1])
            assert info2["iters"] == out[1][3]
        plan.close()
    # with the data pass timed (events around the pass kernel): direct launches
    plan, X, Y = _plan(gb, P, n, dx, dy, k, dt, lam, s=1400, max_iter=300, gtol=1e-7, check_every=4,
                       graphs=1, time_passes=1)
    sig3, U3, V3, info3 = gb.cca_solve(plan)
    assert np.array_equal(np64(sig3), out[1][0])
    assert info3["pass_count"] == info3["iters"] + 1 and info3["pass_ms"] > 0, info3
    plan.close()
    a, b = out[0], out[1]
    assert a[3] == b[3] and a[3] > 8, (a[3], b[3])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert a[4] == b[4], (a[4], b[4])


@pytest.mark.parametrize("dt", ["f64", "bf16"])
def test_ritz_stopping_rule(gb, dt):
    """Option rtol: the Ritz values of span([U, eta]) are recorded at every
    check (GBCCA_Q_RITZ), the last two recorded changes (relative to the
    largest value) are below rtol, the
    solve ends with status OK before max_iter, and the returned correlations
    (the final refinement, one iteration after the last check: the check runs
    beside the rest of its iteration and its verdict ends the solve after it)
    are within rtol of the last recorded values, and the oracle's."""
    n, dx, dy, k, lam = 20000, 96, 72, 5, 1e-3
    P = cca_latent_problem(n, dx, dy, latent=8, noise=0.5, dtype=dt, seed=41,
                           latent_scale=[1.0, 0.8, 0.6, 0.45, 0.3, 0.2, 0.12, 0.07])
    rtol = 1e-9 if dt == "f64" else 1e-7
    plan, _, _ = _plan(gb, P, n, dx, dy, k, dt, lam, max_iter=600, gtol=0.0, rtol=rtol, check_every=4, refine=2)
    sig, U, V, info = gb.cca_solve(plan)
    assert info["status"] == gb.OK and info["iters"] < 600, info
    R = np64(gb.query(plan, gb.Q_RITZ)).reshape(-1, k)
    R = R[np.any(R != 0, axis=1)]
    assert R.shape[0] >= 3
    chg = np.max(np.abs(np.diff(R, axis=0)), axis=1) / np.max(np.abs(R[1:]), axis=1)
    assert chg[-1] < rtol and chg[-2] < rtol, chg[-3:]
    s = np64(sig)
    assert np.max(np.abs(s - R[-1]) / s) < rtol, (s, R[-1])
    ref, _, _ = OC.cca_qr(P["X64"], P["Y64"], lam, lam, k)
    assert rel(s, ref) < (1e-9 if dt == "f64" else 1e-6), (s, ref, info)
