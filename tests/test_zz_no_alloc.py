"""Allocation-free sketch Gram (gbcca_sketch_gram_noalloc) through the C ABI.

Compared with the preconditioner that the existing entry points build:
after gbcca_cca_precondition on an FP64 plan, gbcca_query returns S X and
R_x with R_x^T R_x = (S X)^T (S X) + lambda I; the allocation-free Gram of
the queried S X must reproduce R_x^T R_x.  Two calls in a row must agree
bit for bit (the scratch is reused; its partials are fully rewritten).
This file is collected last so that it also runs after every other test.
"""
import numpy as np
import pytest

from gpu_util import to_dev, np64, rel
from synth import cca_latent_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2106_12060_gb300 as m
    torch.cuda.set_device(0)
    return m


def test_matches_preconditioner_of_existing_entry_point(gb):
    import torch
    n, dx, dy, k, lam, s = 3000, 60, 50, 4, 1e-2, 440
    P = cca_latent_problem(n, dx, dy, latent=6, dtype="f64", seed=11)
    plan = gb.cca_plan(n, dx, dy, k, "f64", gb.default_options(s=s, seed=5, max_iter=2))
    gb.cca_precondition(plan, to_dev(P["X"], "f64"), to_dev(P["Y"], "f64"), lam, lam)
    SX = gb.query(plan, gb.Q_SKETCH_X).reshape(s, dx)
    Rx = np64(gb.query(plan, gb.Q_R_X)).reshape(dx, dx)
    torch.cuda.synchronize()
    # a row stride larger than d exercises lda
    wide = torch.zeros(s, dx + 7, dtype=torch.float64, device="cuda")
    wide[:, :dx] = SX
    A = wide[:, :dx]
    C1 = torch.full((dx, dx), float("nan"), dtype=torch.float64, device="cuda")
    C2 = torch.full((dx, dx), float("nan"), dtype=torch.float64, device="cuda")
    gb.sketch_gram_noalloc(A, lam, C1)
    gb.sketch_gram_noalloc(A, lam, C2)
    torch.cuda.synchronize()
    c1, c2 = np64(C1), np64(C2)
    assert np.array_equal(c1, c2)
    assert rel(c1, Rx.T @ Rx) < 1e-12
    sx = np64(SX)
    assert rel(c1, sx.T @ sx + lam * np.eye(dx)) < 1e-13


def test_largest_d_matches_fp64_gram(gb):
    """d = gbcca_sketch_gram_noalloc_max_d() (one partial slab fills the
    scratch): the result equals the FP64 Gram computed on the host, on two
    calls in a row."""
    import torch
    d = gb.sketch_gram_noalloc_max_d()
    m, lam = 1500, 0.25
    rng = np.random.default_rng(3)
    a = rng.standard_normal((m, d))
    A = torch.from_numpy(a).cuda()
    C1 = torch.full((d, d), float("nan"), dtype=torch.float64, device="cuda")
    C2 = torch.full((d, d), float("nan"), dtype=torch.float64, device="cuda")
    gb.sketch_gram_noalloc(A, lam, C1)
    gb.sketch_gram_noalloc(A, lam, C2)
    torch.cuda.synchronize()
    c1, c2 = np64(C1), np64(C2)
    assert np.array_equal(c1, c2)
    assert rel(c1, a.T @ a + lam * np.eye(d)) < 1e-13


def test_rejects_d_beyond_scratch(gb):
    import torch
    dmax = gb.sketch_gram_noalloc_max_d()
    assert dmax * dmax <= (1 << 20) < (dmax + 1) * (dmax + 1)
    d = dmax + 1
    A = torch.zeros(2, d, dtype=torch.float64, device="cuda")
    C = torch.zeros(d, d, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbccaError) as e:
        gb.sketch_gram_noalloc(A, 0.0, C)
    assert e.value.code == gb.ERR_INVALID_ARG
    assert str(dmax) in str(e.value)
    assert torch.count_nonzero(C).item() == 0
