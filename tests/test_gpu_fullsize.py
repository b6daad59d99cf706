"""Full-size workloads through the C ABI, checked against the FP64 oracle.

The tall CCA workload runs with the benchmark's exact settings (SRHT s=4096,
gtol from bench.py): canonical correlations within 1e-6 relative and the
relative objective suboptimality below 1e-6.  The LDA workload (n=100000,
d=784, 10 classes, FP32): generalized eigenvalues within 1e-6.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel
from oracle.cca import cca_qr, default_mu
from oracle import lda as OL
from synth import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def tall():
    P = make_workload("cca_tall_bf16")
    c = P["config"]
    ref, _, _ = cca_qr(P["X64"], P["Y64"], c["lam"], c["lam"], c["k"])
    return P, ref


@pytest.mark.parametrize("refine", [1, 2])
def test_tall_cca_bench_settings(gb, tall, refine):
    """refine = 1: FP64 Rayleigh-Ritz Grams; refine = 2 (bench.REFINE): from
    the tensor-core pass."""
    import bench
    P, ref = tall
    c = P["config"]
    o = gb.default_options(sketch=gb.SRHT, s=c["s"], seed=c["seed"], max_iter=1000, gtol=bench.GTOL,
                           rtol=bench.RTOL, check_every=bench.CHECK_EVERY, refine=refine)
    plan = gb.cca_plan(c["n"], c["dx"], c["dy"], c["k"], c["dtype"], o)
    X, Y = to_dev(P["X"], c["dtype"]), to_dev(P["Y"], c["dtype"])
    gb.cca_precondition(plan, X, Y, c["lam"], c["lam"])
    sig, U, V, info = gb.cca_solve(plan)
    s = np64(sig)
    assert info["status"] == gb.OK, info
    mu = default_mu(c["k"])
    subopt = abs(np.dot(ref, mu) - np.dot(s, mu)) / np.dot(ref, mu)
    assert subopt < 1e-6, (subopt, info)
    assert rel(s, ref) < 1e-6, (s, ref, info)


def _bench_solve(gb, P, refine):
    import bench
    c = P["config"]
    o = gb.default_options(sketch=gb.SRHT, s=c["s"], seed=c["seed"], max_iter=1000, gtol=bench.GTOL,
                           rtol=bench.RTOL, check_every=bench.CHECK_EVERY, refine=refine)
    plan = gb.cca_plan(c["n"], c["dx"], c["dy"], c["k"], c["dtype"], o)
    X, Y = to_dev(P["X"], c["dtype"]), to_dev(P["Y"], c["dtype"])
    gb.cca_precondition(plan, X, Y, c["lam"], c["lam"])
    sig, U, V, info = gb.cca_solve(plan)
    s = np64(sig)
    plan.close()
    return s, info


@pytest.mark.parametrize("seed", [1, 2])
def test_tall_cca_bench_settings_held_out_seeds(gb, seed):
    """The benchmark's stopping rule (bench.RTOL, bench.REFINE) must hold on
    instances it was not chosen on: other seeds of the data and of the sketch
    reach every correlation within 1e-6 and the relative objective gap below
    1e-6."""
    import bench
    P = make_workload("cca_tall_bf16", seed=seed)
    c = P["config"]
    ref, _, _ = cca_qr(P["X64"], P["Y64"], c["lam"], c["lam"], c["k"])
    s, info = _bench_solve(gb, P, bench.REFINE)
    mu = default_mu(c["k"])
    subopt = abs(np.dot(ref, mu) - np.dot(s, mu)) / np.dot(ref, mu)
    assert info["status"] == gb.OK, info
    assert subopt < 1e-6, (subopt, info)
    assert rel(s, ref) < 1e-6, (s, ref, info)


@pytest.fixture(scope="module")
def mixed():
    P = make_workload("cca_tall_bf16_mixed")
    c = P["config"]
    ref, _, _ = cca_qr(P["X64"], P["Y64"], c["lam"], c["lam"], c["k"])
    return P, ref


def test_tall_cca_haar_mixed(gb, mixed):
    """The tall workload with each view's scaled columns rotated by a
    Haar-random orthogonal matrix (every stored column mixes all scales), at
    the benchmark's settings.  Here the products X U cancel: the sum of
    |terms| is ~300 times the result, and the tensor-core pass's FP32
    accumulation leaves the Grams it returns (Phi^T G) with ~2e-5 relative
    error, which floors the BF16 path near 2e-6 (measured 2.1e-6); the test
    holds it to 3e-6.  The FP64 form on the same values reaches 1e-8
    (next test)."""
    P, ref = mixed
    import bench
    s, info = _bench_solve(gb, P, bench.REFINE)
    assert info["status"] == gb.OK, info
    assert rel(s, ref) < 3e-6, (s, ref, info)


def test_tall_cca_haar_mixed_fp64_storage(gb, mixed):
    P, ref = mixed
    c = P["config"]
    o = gb.default_options(sketch=gb.SRHT, s=c["s"], seed=c["seed"], max_iter=1000, gtol=1e-6)
    plan = gb.cca_plan(c["n"], c["dx"], c["dy"], c["k"], "f64", o)
    gb.cca_precondition(plan, to_dev(P["X64"], "f64"), to_dev(P["Y64"], "f64"), c["lam"], c["lam"])
    sig, U, V, info = gb.cca_solve(plan)
    plan.close()
    assert rel(np64(sig), ref) < 1e-8, (np64(sig), ref, info)


def test_tall_cca_fp64_storage(gb, tall):
    """The plain FP64 form (the same BF16 values stored in FP64, FP64 pass):
    canonical correlations within 1e-8 of the oracle."""
    P, ref = tall
    c = P["config"]
    o = gb.default_options(sketch=gb.SRHT, s=c["s"], seed=c["seed"], max_iter=1000, gtol=1e-6)
    plan = gb.cca_plan(c["n"], c["dx"], c["dy"], c["k"], "f64", o)
    X, Y = to_dev(P["X64"], "f64"), to_dev(P["Y64"], "f64")
    gb.cca_precondition(plan, X, Y, c["lam"], c["lam"])
    sig, U, V, info = gb.cca_solve(plan)
    assert rel(np64(sig), ref) < 1e-8, (np64(sig), ref, info)


@pytest.mark.parametrize("name", ["lda_f32", "lda_f32_mixed"])
def test_lda_workload(gb, name):
    """lda_f32_mixed: within-class covariance Q diag(e) Q^T with Q Haar."""
    import torch
    P = make_workload(name)
    c = P["config"]
    lam = 1e-6 * float(np.trace(OL.scatters(P["X64"], P["y"], c["l"])[1])) / c["d"]
    import bench
    o = gb.default_options(s=c["s"], max_iter=1000, gtol=0.0, rtol=bench.RTOL, check_every=bench.LDA_CHECK_EVERY,
                           refine=bench.LDA_REFINE)
    plan = gb.lda_plan(c["n"], c["d"], c["l"], c["k"], c["dtype"], o)
    X = to_dev(P["X"], c["dtype"])
    y = torch.from_numpy(P["y"]).cuda()
    rho, W, info = gb.lda_solve(plan, X, y, lam)
    ref, _ = OL.lda_geneig(P["X64"], P["y"], c["l"], lam, c["k"])
    assert info["status"] == gb.OK, info
    assert rel(np64(rho), ref) < 1e-6, (np64(rho), ref, info)
