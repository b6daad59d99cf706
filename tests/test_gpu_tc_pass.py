"""GPU parity of the tensor-core (tcgen05 + TMA) fused pass for BF16 data.

The pass rounds Phi to its bf16 hi + lo representation (the point it
evaluates); the expected values use that same rounded Phi.  Remaining error:
(1) the bf16 hi + lo split of W, 2^-17 relative per element, random over
rows; (2) the tensor cores' FP32 accumulation, which does not round to
nearest: every one of the S accumulation steps of a CTA can shrink the
running sum by up to one FP32 ulp (2^-23 relative), a bias of at most
S * 2^-23.  With 128-row tiles, 8 K-steps per tile and the hi and lo halves
of W, S = 16 * (tiles per cluster of two CTAs).  Tolerances: 2e-6 of the
largest entry for the small cases (S <= 48), S * 2^-23 for the full workload
(2048 tiles over at least 64 resident clusters: at most 32 tiles each).
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel
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
    ox, oy, og = OF.cca_pass(P["X64"], P["Y64"], split_round(Px), split_round(Py))
    return (np64(Gx), np64(Gy), np64(Gram)), (ox, oy, og)


@pytest.mark.parametrize("n,dx,dy,k", [(3001, 192, 136, 5), (128, 128, 128, 12), (20000, 512, 384, 10)])
def test_tc_pass_ragged(gb, n, dx, dy, k):
    P = cca_latent_problem(n, dx, dy, latent=6, dtype="bf16", seed=n)
    got, exp = _run(gb, P, n, dx, dy, k)
    for g, e in zip(got, exp):
        assert rel(g, e) < 2e-6


def test_tc_pass_full_workload(gb):
    """The tall workload at full size (n = 262144, dx = dy = 512, k = 10)."""
    P = make_workload("cca_tall_bf16")
    c = P["config"]
    got, exp = _run(gb, P, c["n"], c["dx"], c["dy"], c["k"], seed=3)
    tiles_per_cluster = -(-c["n"] // 128 // 64)
    bound = 16 * tiles_per_cluster * 2.0 ** -23
    for g, e in zip(got, exp):
        assert rel(g, e) < bound
