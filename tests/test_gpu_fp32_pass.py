"""GPU parity of the tensor-core (tcgen05 + TMA) pass for FP32 data, CCA
and FDA, through the C ABI.

Both stream a row-interleaved BF16 hi/lo copy of the data (FDA: of the
class-centred rows; 2n rows: row 2i the hi part of data row i, row 2i + 1 its
lo part; 64-row tiles): Z' = Z_hi + Z_lo with |Z - Z'| <= 2^-17 |Z|
entrywise (z in [2^e, 2^(e+1)): |z - hi| <= 2^(e-8), and rounding that
remainder to 8 bits errs by at most 2^(e-17)), and evaluate Phi' = bf16 hi +
lo of Phi (the point the solver then holds).  Products of BF16 operands are
exact in FP32; the remaining errors are the representation of Z (entering
both products), the bf16 hi + lo split of W (2^-17 |W|) and FP32
accumulation.  Each entry is checked against its own bound gamma * ref, ref
the sum of |terms| (|Z|^T (|Z| |Phi'|); for the Gram (|Z||Phi'|)^T
(|Z||Phi'|)).

CCA (one view per CTA of a 2-CTA cluster; views wider than 512 columns split
over two CTAs of a 4-CTA cluster):
  GEMM 1  d / 16 + 2 FP32 roundings along a chain (two issuers, hi and lo
          columns of Phi), plus the addition of the hi-row and lo-row
          products of the same data row;
  GEMM 2  4 MMAs per 64-row tile, T tiles per cluster, one more addition at
          the drain (hi + lo columns of W);
  reduce  per-cluster partials summed with compensation (<= 2 ulp);
  gamma = 3 * 2^-17 + 2^-23 (2 (d / 16 + 2) + 2 + 2 (4 T + 1) + 4),
T = ceil(ceil(2n / 64) / clusters) with at least min(tiles, 64) clusters.  The
Gram is Phi_bd^T G formed in FP64: the same gamma against |W|^T |W|.

FDA (the one view's 128-column pairs split over the two CTAs of a cluster,
which add their partial W of every tile): the same terms with the chain of
the longer half (d_h = 128 ceil(P / 2) columns, P = ceil(d / 128)) and one
more addition for the halves' sum:
  gamma = 3 * 2^-17 + 2^-23 (2 (d_h / 16 + 2) + 2 + 2 + 2 (4 T + 1) + 4).
Counting every MMA as two FP32 roundings of at most 2^-23 of the running sum.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, bound_ratio, cca_pass_refs, rel
from oracle import fused as OF
from oracle import lda as OL
from oracle.cca import cca_qr
from synth import cca_latent_problem, lda_problem, make_workload, f32_to_bf16_bits, bf16_bits_to_f32

pytestmark = pytest.mark.gpu


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


def gamma_solo(n, d):
    tiles = -(-2 * n // 64)
    T = -(-tiles // min(tiles, 64))
    dh = 128 * -(-(-(-d // 128)) // 2)
    return 3 * 2.0 ** -17 + 2.0 ** -23 * (2 * (dh / 16 + 2) + 2 + 2 + 2 * (4 * T + 1) + 4)


def gamma_interleaved(n, d):
    tiles = -(-2 * n // 64)
    T = -(-tiles // min(tiles, 64))
    return 3 * 2.0 ** -17 + 2.0 ** -23 * (2 * (d / 16 + 2) + 2 + 2 * (4 * T + 1) + 4)


def _check(got, exp, refs, gamma):
    for name, g, e, r in zip(("G", "G2", "Gram"), got, exp, refs):
        if g is None:
            continue
        ratio = bound_ratio(g, e, r, gamma)
        assert ratio <= 1.0, (name, ratio, gamma)


def _cca(gb, P, n, dx, dy, k, seed=0):
    import torch
    plan = gb.cca_plan(n, dx, dy, k, "f32", gb.default_options(warm_start=0))
    X, Y = to_dev(P["X"], "f32"), to_dev(P["Y"], "f32")
    gb.cca_precondition(plan, X, Y, 1e-2, 1e-2)
    rng = np.random.default_rng(seed)
    Px = rng.standard_normal((dx, 2 * k)) / np.sqrt(dx)
    Py = rng.standard_normal((dy, 2 * k)) / np.sqrt(dy)
    Gx, Gy, Gram = gb.fused_pass(plan, torch.from_numpy(Px).cuda(), torch.from_numpy(Py).cuda())
    torch.cuda.synchronize()
    Pxr, Pyr = split_round(Px), split_round(Py)
    exp = OF.cca_pass(P["X64"], P["Y64"], Pxr, Pyr)
    rx, ry, rg, _ = cca_pass_refs(P["X64"], P["Y64"], Pxr, Pyr)
    plan.close()
    return (np64(Gx), np64(Gy), np64(Gram)), exp, (rx, ry, rg)


@pytest.mark.parametrize("n,dx,dy,k", [(3001, 192, 136, 5), (4099, 70, 45, 5), (20000, 512, 384, 10),
                                       (64, 64, 40, 1), (33, 24, 8, 3), (12345, 500, 24, 12), (7001, 136, 97, 15),
                                       (3001, 768, 136, 6)])
def test_fp32_cca_pass_ragged(gb, n, dx, dy, k):
    P = cca_latent_problem(n, dx, dy, latent=6, dtype="f32", seed=n, colscale=(1.0, 1e-3))
    got, exp, refs = _cca(gb, P, n, dx, dy, k)
    _check(got, exp, refs, gamma_interleaved(n, max(dx, dy)))


def test_fp32_cca_pass_full_workload(gb):
    """The tall workload stored in FP32 (n = 262144, dx = dy = 512, k = 10)."""
    P = make_workload("cca_tall_f32")
    c = P["config"]
    got, exp, refs = _cca(gb, P, c["n"], c["dx"], c["dy"], c["k"], seed=3)
    _check(got, exp, refs, gamma_interleaved(c["n"], 512))


def _lda(gb, P, n, d, l, k, seed=0):
    import torch
    plan = gb.lda_plan(n, d, l, k, "f32", gb.default_options(max_iter=1))
    X = to_dev(P["X"], "f32")
    y = torch.from_numpy(P["y"]).cuda()
    gb.lda_solve(plan, X, y, 1e-2)
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((d, 2 * k)) / np.sqrt(d)
    G, _, Gram = gb.fused_pass(plan, torch.from_numpy(Phi).cuda())
    torch.cuda.synchronize()
    Pr = split_round(Phi)
    eg, egram = OF.lda_pass(P["X64"], P["y"], l, Pr)
    _, _, _, _, Xhat = OL.class_stats(P["X64"], P["y"], l)
    aP = np.abs(Xhat) @ np.abs(Pr)
    plan.close()
    return (np64(G), None, np64(Gram)), (eg, None, egram), (np.abs(Xhat).T @ aP, None, aP.T @ aP)


# ragged rows and columns; one pair (the second CTA then streams an empty
# pair); 2k = 26 (two column groups); a 1024-column view
@pytest.mark.parametrize("n,d,l,k", [(5003, 61, 6, 5), (20000, 784, 10, 9), (257, 130, 3, 2), (6001, 200, 16, 13),
                                     (3001, 1024, 5, 4)])
def test_fda_pass_ragged(gb, n, d, l, k):
    P = lda_problem(n, d, l, dtype="f32", seed=n)
    got, exp, refs = _lda(gb, P, n, d, l, k)
    _check(got, exp, refs, gamma_solo(n, d))


def test_fda_pass_full_workload(gb):
    """The LDA workload (n = 100000, d = 784, 10 classes, k = 9)."""
    P = make_workload("lda_f32")
    c = P["config"]
    got, exp, refs = _lda(gb, P, c["n"], c["d"], c["l"], c["k"], seed=4)
    _check(got, exp, refs, gamma_solo(c["n"], c["d"]))


def test_tall_f32_solve(gb):
    """The tall workload stored in FP32, solved with the benchmark's settings
    on the tensor-core pass: every correlation within 1e-6 of the oracle."""
    import bench
    P = make_workload("cca_tall_f32")
    c = P["config"]
    ref, _, _ = cca_qr(P["X64"], P["Y64"], c["lam"], c["lam"], c["k"])
    o = gb.default_options(sketch=gb.SRHT, s=c["s"], seed=c["seed"], max_iter=1000, gtol=bench.GTOL,
                           rtol=bench.RTOL, check_every=bench.CHECK_EVERY, refine=bench.REFINE)
    plan = gb.cca_plan(c["n"], c["dx"], c["dy"], c["k"], "f32", o)
    gb.cca_precondition(plan, to_dev(P["X"], "f32"), to_dev(P["Y"], "f32"), c["lam"], c["lam"])
    sig, U, V, info = gb.cca_solve(plan)
    assert info["status"] == gb.OK, info
    assert rel(np64(sig), ref) < 1e-6, (np64(sig), ref, info)


def test_wait_bound_reports_timeout_and_context_survives(gb):
    """A pipeline-wait bound of one cycle makes the first wait of the FDA
    tensor-core pass run out: every CTA drains its own copies and MMAs and
    leaves, and the solve returns GBCCA_ERR_TIMEOUT (no hang, no fault).  A
    plan with the default bound then solves the same data correctly."""
    import torch
    n, d, l, k, lam = 6000, 96, 5, 4, 1e-2
    P = lda_problem(n, d, l, dtype="f32", seed=31)
    X = to_dev(P["X"], "f32")
    y = torch.from_numpy(P["y"]).cuda()
    plan = gb.lda_plan(n, d, l, k, "f32", gb.default_options(wait_cycles=1, max_iter=50))
    with pytest.raises(gb.GbccaError) as e:
        gb.lda_solve(plan, X, y, lam)
    assert e.value.code == gb.ERR_TIMEOUT, str(e.value)
    torch.cuda.synchronize()
    plan.close()
    plan = gb.lda_plan(n, d, l, k, "f32", gb.default_options(max_iter=2000, gtol=0.0, rtol=1e-7))
    rho, _, info = gb.lda_solve(plan, X, y, lam)
    ref, _ = OL.lda_geneig(P["X64"], P["y"], l, lam, k)
    assert info["status"] == gb.OK, info
    assert rel(np64(rho), ref) < 1e-6, (np64(rho), ref)
    plan.close()


def test_bad_labels_are_rejected(gb):
    """A label outside [0, n_classes) is refused before any kernel indexes a
    class table with it."""
    import torch
    n, d, l, k = 500, 12, 3, 2
    P = lda_problem(n, d, l, dtype="f32", seed=2)
    y = P["y"].copy()
    y[17] = l
    plan = gb.lda_plan(n, d, l, k, "f32", gb.default_options())
    with pytest.raises(gb.GbccaError) as e:
        gb.lda_solve(plan, to_dev(P["X"], "f32"), torch.from_numpy(y).cuda(), 1e-2)
    assert e.value.code == gb.ERR_INVALID_ARG and "label" in str(e.value)
    plan.close()
