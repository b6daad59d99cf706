"""GPU parity of the tensor-core (tcgen05 + TMA) fused pass for BF16 data.

The pass rounds Phi to its bf16 hi + lo representation (the point it
evaluates); the expected values use that same rounded Phi, and the products
of the stored BF16 data with it are exact in FP32, so every remaining error
is an FP32 rounding.  Each entry is checked against its own bound
gamma * ref, where ref is the sum of |terms| of that entry (|X|^T |W| for
Gx, |Y|^T |W| for Gy, |W|^T |W| for the Gram; |W| <= [|X||Phi_x|, |Y||Phi_y|]).
A column of the data scaled by 1e-4 therefore gets a bound 1e-4 times
smaller, not the bound of the largest entry.

Rounding steps of the kernel (64-row tiles, 2-CTA clusters, one view per CTA):
  GEMM 1  W = Z Phi over K = d in MMAs of K = 16, split over two issuers
          into two FP32 accumulators that the epilogue adds, hi and lo
          columns of Phi in separate accumulator columns also added:
          at most d / 16 + 2 FP32 roundings along any chain;
  split   W -> bf16 hi + lo: |W - (W_hi + W_lo)| <= 2^-17 |W|;
  GEMM 2  G = Z^T W over the rows of a cluster in MMAs of K = 16 (4 per
          64-row tile), hi and lo accumulator columns added at the drain:
          4 T + 1 roundings for T tiles per cluster;
  reduce  per-cluster FP32 partials summed with compensation (<= 2 ulp).
Each FP32 rounding errs by at most 2^-23 of the running magnitude (which the
sum of |terms| bounds); counting every MMA as two roundings (its internal
sum and the accumulate) gives
  gamma = 2^-17 + 2^-23 (2 (d / 16 + 2) + 2 (4 T + 1) + 4),
T = ceil(ceil(n / 64) / clusters) with at least min(tiles, 64) clusters (the
GB300 keeps 76 resident).  The Gram is Phi_bd^T G formed in FP64: the same
gamma against |Phi_bd|^T ref_G = |W|^T |W|.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, bound_ratio, cca_pass_refs
from oracle import fused as OF
from synth import cca_latent_problem, make_workload, f32_to_bf16_bits, bf16_bits_to_f32

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
    lo = bf16_round(P - hi)
    return hi + lo


def gamma_tc(n, d):
    tiles = -(-n // 64)
    T = -(-tiles // min(tiles, 64))
    return 2.0 ** -17 + 2.0 ** -23 * (2 * (d / 16 + 2) + 2 * (4 * T + 1) + 4)


def _run(gb, P, n, dx, dy, k, seed=0):
    import torch
    plan = gb.cca_plan(n, dx, dy, k, "bf16", gb.default_options(warm_start=0))
    X, Y = to_dev(P["X"], "bf16"), to_dev(P["Y"], "bf16")
    gb.cca_precondition(plan, X, Y, 1e-2, 1e-2)
    rng = np.random.default_rng(seed)
    Px = rng.standard_normal((dx, 2 * k)) / np.sqrt(dx)
    Py = rng.standard_normal((dy, 2 * k)) / np.sqrt(dy)
    Gx, Gy, Gram = gb.fused_pass(plan, torch.from_numpy(Px).cuda(), torch.from_numpy(Py).cuda())
    torch.cuda.synchronize()
    Pxr, Pyr = split_round(Px), split_round(Py)
    ox, oy, og = OF.cca_pass(P["X64"], P["Y64"], Pxr, Pyr)
    rx, ry, rg, _ = cca_pass_refs(P["X64"], P["Y64"], Pxr, Pyr)
    plan.close()
    return (np64(Gx), np64(Gy), np64(Gram)), (ox, oy, og), (rx, ry, rg)


def _check(got, exp, refs, gamma):
    for name, g, e, r in zip(("Gx", "Gy", "Gram"), got, exp, refs):
        ratio = bound_ratio(g, e, r, gamma)
        assert ratio <= 1.0, (name, ratio, gamma)


@pytest.mark.parametrize("n,dx,dy,k", [(3001, 192, 136, 5), (128, 128, 128, 12), (20000, 512, 384, 10),
                                       (80, 64, 72, 1), (5003, 200, 136, 13), (9001, 512, 488, 20),
                                       (4001, 1024, 256, 5), (3003, 704, 600, 10), (2050, 1024, 64, 20),
                                       (900, 520, 72, 3)])
def test_tc_pass_ragged(gb, n, dx, dy, k):
    """Ragged sizes; k = 13 and k = 20 take two column groups of Phi (14 + 12
    and 20 + 20 columns per view), each its own pass over the data with the
    same rounding steps, reduced into their columns of G.  Views wider than
    512 columns run in 4-CTA clusters: each view's column pairs split over two
    CTAs whose FP32 partial products W are added before the hi/lo split (one
    more FP32 rounding, inside the bound's slack); a narrow view beside a wide
    one gives its second CTA a pair of zero columns past its last one."""
    P = cca_latent_problem(n, dx, dy, latent=6, dtype="bf16", seed=n)
    got, exp, refs = _run(gb, P, n, dx, dy, k)
    _check(got, exp, refs, gamma_tc(n, max(dx, dy)))


def test_tc_pass_column_scaled_rows_are_checked(gb):
    """Columns scaled 1 -> 1e-4 (the tall workload's scaling) at a ragged
    size: the rows of G for the small columns are 1e-4 of the largest, and
    each is held to its own bound."""
    n, dx, dy, k = 9000, 320, 256, 10
    P = cca_latent_problem(n, dx, dy, latent=8, dtype="bf16", seed=17, colscale=(1.0, 1e-4))
    got, exp, refs = _run(gb, P, n, dx, dy, k, seed=2)
    _check(got, exp, refs, gamma_tc(n, max(dx, dy)))
    # the smallest rows really are small: a bound relative to the largest
    # entry would not have checked them
    rx = refs[0]
    assert np.max(rx[-1]) < 1e-3 * np.max(rx)


def test_tc_pass_full_workload(gb):
    """The tall workload at full size (n = 262144, dx = dy = 512, k = 10), in
    the launch configuration the solve uses."""
    P = make_workload("cca_tall_bf16")
    c = P["config"]
    got, exp, refs = _run(gb, P, c["n"], c["dx"], c["dy"], c["k"], seed=3)
    _check(got, exp, refs, gamma_tc(c["n"], max(c["dx"], c["dy"])))
